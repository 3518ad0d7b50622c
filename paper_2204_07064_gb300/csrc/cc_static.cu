// One cached Conv1d step that allocates no device memory.
//
// Some callers of this library cannot allocate device memory when they want
// to run a layer: a real-time audio callback (a DSP thread may not block, and
// cudaMalloc can synchronise the device and take an unbounded time, which
// the host hears as a dropout), or a plug-in embedded in a host that hands it
// a fixed, pre-reserved memory budget.  This entry point serves them: the
// caller passes its input, weights, cached frames and output, and every
// intermediate buffer (packed weights and the window of cached frames
// followed by the new buffer) lives in one file-scope device array reserved
// when the library is loaded.  The arithmetic is the library's FP32 cached
// convolution kernel, unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/cachedconv.h"
#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {
namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;  // the documented maximum: 16 MiB
constexpr size_t kHeaderBytes = 256;               // slot index (int32) + step counter (int64)
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Host-side addresses of the array, one per device (the array's name in host
// code is only a stand-in and must not be passed to a kernel).
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cc_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(CC_ERR_CUDA, "no current CUDA device for the static scratch");
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(CC_ERR_CUDA, "cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CC_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Header (slot 0, zero steps), a copy of the bias (the convolution kernel
// reads it four channels at a time, so it must be 16-byte aligned, which a
// caller's pointer into a packed parameter buffer need not be), weights
// repacked [c_out][c_in][K] -> [c_out][K][c_in], and the window ring: cached
// frames at times -hist..-1 (rows R-hist..R-1), the new buffer at times
// 0..n-1 (rows 0..n-1).
__global__ void k_static_prepare(unsigned char* scratch, size_t b_off, size_t w_off, size_t win_off,
                                 const float* x, int64_t n, int32_t cin, int32_t cout, int32_t K,
                                 const float* w, const float* bias, const float* cache, int32_t hist) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    *reinterpret_cast<int32_t*>(scratch) = 0;
    *reinterpret_cast<int64_t*>(scratch + 8) = 0;
  }
  if (bias) {
    float* B = reinterpret_cast<float*>(scratch + b_off);
    for (int64_t i = tid; i < cout; i += stride) B[i] = bias[i];
  }
  float* A = reinterpret_cast<float*>(scratch + w_off);
  const int64_t nw = (int64_t)cout * cin * K;
  for (int64_t i = tid; i < nw; i += stride) {
    const int64_t o = i / ((int64_t)K * cin);
    const int64_t r = i - o * K * cin;
    const int64_t k = r / cin, c = r - k * cin;
    A[i] = w[(o * cin + c) * K + k];
  }
  float* win = reinterpret_cast<float*>(scratch + win_off);
  const int64_t rows = hist + n;
  for (int64_t i = tid; i < rows * cin; i += stride) {
    const int64_t row = i / cin, c = i - row * cin;
    if (row < n)
      win[i] = x[row * cin + c];
    else
      win[i] = cache[(row - n) * cin + c];  // time row - rows, i.e. -hist .. -1
  }
}

// New cached frames: times n-hist .. n-1 of the window.
__global__ void k_static_update_cache(const unsigned char* scratch, size_t win_off, int64_t n,
                                      int32_t cin, int32_t hist, float* cache) {
  const float* win = reinterpret_cast<const float*>(scratch + win_off);
  const int64_t rows = hist + n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)hist * cin;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = i / cin, c = i - q * cin;
    int64_t t = n - hist + q;
    if (t < 0) t += rows;
    cache[i] = win[t * cin + c];
  }
}

int grid_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

}  // namespace
}  // namespace cc

extern "C" cc_status cc_cached_conv1d_static(const float* x, int64_t n, int32_t c_in, int32_t c_out,
                                             int32_t kernel, int32_t dilation, int32_t pad_left,
                                             int32_t pad_right, int32_t act_in, const float* weight,
                                             const float* bias, float* cache, float* y,
                                             void* cuda_stream) {
  using namespace cc;
  if (n < 0 || c_in <= 0 || c_out <= 0 || kernel <= 0 || dilation <= 0 || pad_left < 0 || pad_right < 0)
    return fail(CC_ERR_INVALID_ARG, "bad layer geometry");
  if (act_in != CC_ACT_NONE && act_in != CC_ACT_LEAKY) return fail(CC_ERR_INVALID_ARG, "bad activation");
  const int64_t hist = (int64_t)pad_left + pad_right;
  if ((int64_t)(kernel - 1) * dilation > hist)
    return fail(CC_ERR_INVALID_ARG, "kernel span exceeds the padding: the layer cannot stream");
  // the device's copy of the array is looked up before the empty-buffer
  // return, so that a call with n == 0 is a warm-up that does the set-up
  unsigned char* scratch = nullptr;
  cc_status s = scratch_for_current_device(&scratch);
  if (s) return s;
  if (n == 0) return CC_OK;
  if (!x || !weight || !y || (hist > 0 && !cache)) return fail(CC_ERR_INVALID_ARG, "null buffer");
  const size_t w_bytes = (size_t)c_out * c_in * kernel * sizeof(float);
  const size_t win_bytes = (size_t)(hist + n) * c_in * sizeof(float);
  const size_t b_off = kHeaderBytes;
  const size_t w_off = b_off + align256((size_t)c_out * sizeof(float));
  const size_t win_off = align256(w_off + w_bytes);
  const size_t need = win_off + align256(win_bytes);
  if (need > kStaticScratchBytes || hist + n > INT32_MAX)
    return fail(CC_ERR_INVALID_ARG,
                "layer needs %zu bytes of scratch (packed weights + %lld-frame window); the static "
                "scratch holds %zu bytes",
                need, (long long)(hist + n), kStaticScratchBytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int64_t prep_work = std::max<int64_t>((int64_t)c_out * c_in * kernel, (hist + n) * c_in);
  k_static_prepare<<<grid_for(prep_work), 256, 0, st>>>(scratch, b_off, w_off, win_off, x, n, c_in, c_out,
                                                         kernel, weight, bias, cache, (int32_t)hist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ERR_CUDA, "prepare launch failed: %s", cudaGetErrorString(e));

  ConvArgs a{};
  a.A = reinterpret_cast<const float*>(scratch + w_off);
  a.bias = bias ? reinterpret_cast<const float*>(scratch + b_off) : nullptr;
  a.M = c_out;
  a.Kt = kernel * c_in;
  a.taps = kernel;
  a.cin = c_in;
  a.dil = dilation;
  a.stride = 1;
  a.hist = (int32_t)hist;
  a.ncols = (int32_t)n;
  a.act = act_in;
  a.cout = c_out;
  a.phases = 1;
  a.out_u = (int32_t)n;
  a.in.off = (int64_t)win_off;
  a.in.rows = (int32_t)(hist + n);
  a.in.chans = c_in;
  a.in.u = (int32_t)n;
  a.in.dtype = kDtF32;
  a.out.ext = y;
  a.out.ext_stride = n * c_out;
  a.batch.arena = reinterpret_cast<char*>(scratch);
  a.batch.slot_bytes = 0;
  a.batch.slots = reinterpret_cast<const int32_t*>(scratch);
  a.batch.counters = reinterpret_cast<const int64_t*>(scratch + 8);
  a.batch.seeds = nullptr;
  a.batch.count = 1;
  e = launch_conv_f32(a, st);
  if (e != cudaSuccess) return fail(CC_ERR_CUDA, "conv launch failed: %s", cudaGetErrorString(e));
  if (hist > 0) {
    k_static_update_cache<<<grid_for(hist * c_in), 256, 0, st>>>(scratch, win_off, n, c_in,
                                                                  (int32_t)hist, cache);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, "cache update launch failed: %s", cudaGetErrorString(e));
  }
  return CC_OK;
}
