// Allocation-free variant of the FSM inverse Laplace transform (bem_fsm_eval_noalloc).
//
// Who needs it: code that must not allocate device memory while it runs -- for example a caller
// that works inside a fixed memory budget handed to it by a host application or a memory pool
// it does not own, a real-time loop where a cudaMalloc could stall on a device-wide
// synchronisation, or a plug-in that is only given device buffers and a stream.  Such a caller
// cannot create a bem_ctx (contexts allocate their working memory), so this entry point takes
// only device pointers and a stream and uses no memory of its own beyond one fixed scratch
// array.
//
// The scratch (the nt x nc phase table of the transform) is a file-scope __device__ array of
// kNoAllocTable complex doubles (4 MiB).  Every GPU on which the library is loaded holds it for
// the life of the process.  In host code the array's name is only a host-side stand-in, so its
// device address is obtained once per device with cudaGetSymbolAddress (with that device
// current) and cached; the first call on a device performs that set-up and should therefore come
// before any stream capture.  All calls share the array and it keeps the last call's contents;
// the transform overwrites every entry it reads, so nothing needs clearing.  Calls that overlap
// on the GPU (other streams, other host threads on the same device) race on the array.
#include <mutex>

#include "kernel_math.cuh"

namespace bem {

constexpr int64_t kNoAllocTable = int64_t(1) << 18;  // complex doubles: nt * nc <= 262144
constexpr int kMaxDevices = 64;

static __device__ __align__(256) cx<double> g_fsm_scratch[kNoAllocTable];

namespace {
std::mutex g_mu;
cx<double>* g_scratch_addr[kMaxDevices] = {nullptr};
thread_local std::string g_err;  // per calling thread, so the returned pointer stays valid

cx<double>* scratch_for(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    BEM_CUDA(cudaGetSymbolAddress(&p, g_fsm_scratch));
    g_scratch_addr[dev] = static_cast<cx<double>*>(p);
  }
  return g_scratch_addr[dev];
}

void require_device_ptr(const void* p, int dev, const char* name) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    throw Error(BEM_ERR_INVALID_ARG, std::string(name) + " is not a device pointer");
  }
  if (!(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ||
      (at.type == cudaMemoryTypeDevice && at.device != dev))
    throw Error(BEM_ERR_INVALID_ARG,
                std::string(name) + " must be device memory of the current device");
}
}  // namespace

}  // namespace bem

extern "C" const char* bem_noalloc_last_error(void) { return bem::g_err.c_str(); }

extern "C" int bem_fsm_eval_noalloc(const double* h, int64_t nc, int64_t m, double eta,
                                    double period, const double* t, int64_t nt, int window,
                                    double* out, void* cuda_stream) {
  using namespace bem;
  try {
    BEM_REQUIRE(h && t && out, "null pointer");
    fsm_check_args(nc, m, eta, period, nt, window);
    if (nt * nc > kNoAllocTable)
      throw Error(BEM_ERR_INVALID_ARG,
                  "nt * nc = " + std::to_string(nt * nc) + " exceeds the fixed scratch of " +
                      std::to_string(kNoAllocTable) + " phase-table entries");
    int dev = 0;
    BEM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error(BEM_ERR_INVALID_ARG, "device index too large");
    require_device_ptr(h, dev, "h");
    require_device_ptr(t, dev, "t");
    require_device_ptr(out, dev, "out");
    cx<double>* table = scratch_for(dev);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    fsm_launch(reinterpret_cast<const cx<double>*>(h), nc, m, eta, period, t, nt, window, out,
               table, st);
    BEM_CUDA(cudaStreamSynchronize(st));
    return BEM_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  }
}
