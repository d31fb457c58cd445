// tomo_oc_step_noalloc: the optimality-criteria update for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to call cudaMalloc at all: runtimes that hand out every byte
// of device memory through their own pool and forbid driver allocations behind their back,
// and latency-critical loops where an allocation's implicit device synchronisation is
// unacceptable.  This entry point needs no grid handle (creating one allocates) and no
// staging buffers: its scratch lives in the file-scope array below, which every GPU that
// loads this library keeps until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"
#include "host.h"

namespace tomo {
extern thread_local std::string g_create_err;
}

namespace {

// Largest design vector accepted (elements).  The scratch holds the per-block candidate
// volumes of the multiplier search (one row of 32 doubles per 2048 elements), the block
// maxima of the final pass, the bracket and the change: about 0.5 MiB in total.
constexpr long long kNoAllocMaxElements = 1LL << 22;  // 4,194,304
constexpr int kNoAllocPartials = (int)((kNoAllocMaxElements + 2047) / 2048) * 32;
constexpr int kNoAllocScalars = 8;  // [0] counter (as unsigned), [2..3] bracket, [1] change

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + kNoAllocScalars];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

tomo_status noalloc_fail(tomo_status st, const char* msg) {
  tomo::g_create_err = msg;
  return st;
}

// p is device (or managed) memory of device dev: the kernels run on the current device and
// read the arrays without peer access, so memory of another GPU is rejected here.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" tomo_status tomo_oc_step_noalloc(int64_t n_el, double h, const float* z,
                                            const float* dcdz, const float* dvdz,
                                            double volfrac, double move, float* z_new,
                                            double* change, void* stream) {
  if (n_el < 1 || n_el > kNoAllocMaxElements)
    return noalloc_fail(TOMO_EINVAL,
                        "tomo_oc_step_noalloc: n_el must be in [1, 4194304] (the size of the "
                        "library's static scratch)");
  if (!(h > 0.0) || !(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0))
    return noalloc_fail(TOMO_EINVAL, "tomo_oc_step_noalloc: need h > 0, 0 < volfrac <= 1, "
                                     "move > 0");
  if (!z || !dcdz || !dvdz || !z_new)
    return noalloc_fail(TOMO_EINVAL, "tomo_oc_step_noalloc: null array");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(TOMO_ECUDA, "tomo_oc_step_noalloc: no usable CUDA device");
  }
  if (!on_device(z, dev) || !on_device(dcdz, dev) || !on_device(dvdz, dev) ||
      !on_device(z_new, dev) || (change && !on_device(change, dev)))
    return noalloc_fail(TOMO_EINVAL,
                        "tomo_oc_step_noalloc: all arrays (and change, if given) must be "
                        "device memory of the current device");
  if (stream) {
    int sdev = -1;
    if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return noalloc_fail(TOMO_EINVAL, "tomo_oc_step_noalloc: invalid stream");
    }
    if (sdev != dev)
      return noalloc_fail(TOMO_EINVAL,
                          "tomo_oc_step_noalloc: the stream belongs to another device");
  }
  if (z_new == z || z_new == dcdz || z_new == dvdz)
    return noalloc_fail(TOMO_EINVAL, "tomo_oc_step_noalloc: z_new overlaps an input");
  double* scratch = nullptr;
  {
    // First call on a device: resolve the device address of the static scratch with that
    // device current.  This must not happen during stream capture.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(TOMO_ECUDA, "tomo_oc_step_noalloc: cudaGetSymbolAddress failed");
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* partials = scratch;
  double* scal = scratch + kNoAllocPartials;
  unsigned* counter = reinterpret_cast<unsigned*>(scal);  // scal[0]
  double* change_dev = scal + 1;
  double* bracket = scal + 2;
  // the grid-completion counter must start at zero; the rest (bracket included: the first
  // pass of the search starts from the full range) is written before it is read
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(double), st);
  const int n = (int)n_el;
  if (e == cudaSuccess && tomo::oc_max_blocks(n) * 32 > kNoAllocPartials) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    const double vmax = volfrac * (double)n_el * h * h * h;
    e = tomo::launch_oc<float>(st, n, z, dcdz, dvdz, vmax, move, z_new, partials, counter,
                               bracket, change_dev, tomo::oc_max_blocks(n));
  }
  if (e == cudaSuccess && change)
    e = cudaMemcpyAsync(change, change_dev, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    std::string msg = std::string("tomo_oc_step_noalloc: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return noalloc_fail(TOMO_ECUDA, msg.c_str());
  }
  return TOMO_OK;
}
