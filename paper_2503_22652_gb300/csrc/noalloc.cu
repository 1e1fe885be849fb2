// rchfsi_filter_step_tf32_static: one TF32 step of the filter recurrence that allocates no device
// memory.  The paper has no counterpart; this exists for callers that must not allocate.
//
// The step is the split-K tcgen05 product of tc_gemm.cu.  Its partial sums, which the regular
// path keeps in a per-handle cudaMalloc'd buffer, live here in a file-scope __device__ array of
// fixed size, so every GPU that loads the library holds RCHFSI_STATIC_SCRATCH_FLOATS floats
// (16 MiB) until the process exits.  Host code cannot use the array's name as a device address
// (it names a host-side shadow), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
#include <mutex>
#include <string>

#include "tc_gemm.cuh"

namespace rchfsi {
void set_last_error(const std::string& msg);  // abi.cu

namespace {

constexpr size_t kScratchFloats = RCHFSI_STATIC_SCRATCH_FLOATS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_splitk_scratch[kScratchFloats];
static __device__ __align__(256) int g_step_flag[4];

struct DeviceAddrs {
  bool ready = false;
  float* scratch = nullptr;
  int* flag = nullptr;
  int sms = 0;
};

std::mutex g_mu;
DeviceAddrs g_dev[kMaxDevices];

// Device addresses of the static arrays on the current device (looked up on first use).
DeviceAddrs device_addrs() {
  int dev = 0;
  RC_CUDA(cudaGetDevice(&dev));
  RC_CHECK(dev >= 0 && dev < kMaxDevices, RCHFSI_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceAddrs& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    RC_CUDA(cudaGetSymbolAddress(&p, g_splitk_scratch));
    d.scratch = static_cast<float*>(p);
    RC_CUDA(cudaGetSymbolAddress(&p, g_step_flag));
    d.flag = static_cast<int*>(p);
    RC_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    d.ready = true;
  }
  return d;
}

// True for memory the current device `dev` can use as a kernel argument: its own device memory, or
// managed memory.  Device memory of another GPU is refused (its address would reach the TMA maps).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Byte range [lo, hi) covered by an m x n column-major FP32 block of leading dimension ld.
struct Span {
  uintptr_t lo, hi;
};
Span block_span(const float* p, int64_t m, int64_t n, int64_t ld) {
  const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
  return {lo, lo + (uintptr_t)(((n - 1) * ld + m) * (int64_t)sizeof(float))};
}
bool overlap(const Span& a, const Span& b) { return a.lo < b.hi && b.lo < a.hi; }

}  // namespace
}  // namespace rchfsi

using namespace rchfsi;

extern "C" int rchfsi_filter_step_tf32_static(const float* A, int64_t lda, const float* Ry, const float* Rx,
                                              const float* W, const double* lambda_y, float a, float b, float c,
                                              int64_t m, int64_t n, int64_t ldr, float* out, void* cuda_stream) {
  try {
    RC_CHECK(m > 0 && n > 0, RCHFSI_ERR_INVALID_ARG, "m and n must be positive");
    RC_CHECK(lda >= m && ldr >= m && (lda * 4) % 16 == 0 && (ldr * 4) % 16 == 0, RCHFSI_ERR_INVALID_ARG,
             "lda and ldr must be >= m and multiples of 4 (16-byte rows)");
    RC_CHECK(A && Ry && out && lambda_y, RCHFSI_ERR_INVALID_ARG, "A, Ry, lambda_y and out are required");
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    RC_CHECK(on_device(A, dev) && on_device(Ry, dev) && on_device(out, dev) && (!Rx || on_device(Rx, dev)) &&
                 (!W || on_device(W, dev)) && on_device(lambda_y, dev),
             RCHFSI_ERR_INVALID_ARG, "every array must be device (or managed) memory of the current device");
    // out is written while Ry and W are still read by other threads: it may coincide with Rx (each
    // element is read before it is written by the same thread) but must not overlap Ry, W or part
    // of Rx
    const Span so = block_span(out, m, n, ldr);
    RC_CHECK(!overlap(so, block_span(Ry, m, n, ldr)) && (!W || !overlap(so, block_span(W, m, n, ldr))) &&
                 (!Rx || Rx == out || !overlap(so, block_span(Rx, m, n, ldr))),
             RCHFSI_ERR_INVALID_ARG, "out may coincide with Rx but must not overlap Ry, W or part of Rx");
    const DeviceAddrs d = device_addrs();
    const size_t need = tc_gemm_tf32_split_floats(d.sms, m, n, m);
    RC_CHECK(need <= kScratchFloats, RCHFSI_ERR_INVALID_ARG,
             "problem needs " + std::to_string(need) + " floats of split-K scratch; the static limit is " +
                 std::to_string(kScratchFloats) + " (RCHFSI_STATIC_SCRATCH_FLOATS)");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    RC_CUDA(cudaMemsetAsync(d.flag, 0, sizeof(int), s));  // the timeout flag must start at zero
    TcRecur r{a, b, c, Ry, Rx, W, lambda_y, out};
    tc_gemm_tf32_recur_ws(s, d.sms, m, n, m, A, lda, Ry, ldr, d.scratch, kScratchFloats, r, ldr, d.flag);
    int flag = 0;
    RC_CUDA(cudaMemcpyAsync(&flag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    if (flag) {
      set_last_error("a bounded wait in the tensor-core kernel ran out");
      return RCHFSI_ERR_TIMEOUT;
    }
    return RCHFSI_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return RCHFSI_ERR_CUDA;
  }
}
