// Shared device/host helpers of the gbcca library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <atomic>
#include <string>
#include <type_traits>

#include "../../include/gbcca.h"

namespace gbcca {

// ---------------------------------------------------------------- errors
void set_last_error(const std::string& msg);
extern std::atomic<long long> g_launches;  // kernels launched by this library

// Device bytes allocated by this thread through counted_malloc since the
// counter was last reset (a plan's workspace is counted while it is made).
inline thread_local int64_t g_alloc_bytes = 0;
inline cudaError_t counted_malloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_alloc_bytes += (int64_t)bytes;
  return e;
}

struct Status {
  int code = GBCCA_OK;
  bool ok() const { return code == GBCCA_OK; }
};

#define GB_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::gbcca::set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
      return GBCCA_ERR_CUDA;                                                              \
    }                                                                                     \
  } while (0)

#define GB_CHECK_LAUNCH()                                                                 \
  do {                                                                                    \
    ::gbcca::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess) {                                                              \
      ::gbcca::set_last_error(std::string("kernel launch at ") + __FILE__ + ":" +          \
                              std::to_string(__LINE__) + ": " + cudaGetErrorString(e_));  \
      return GBCCA_ERR_CUDA;                                                              \
    }                                                                                     \
  } while (0)

#define GB_TRY(expr)           \
  do {                         \
    int r_ = (expr);           \
    if (r_ != GBCCA_OK) return r_; \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Records a timing event on `st`; while `st` is being captured into a CUDA
// graph the record becomes an event-record node of the graph (recorded at
// every replay).
inline cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, st);
}

// Codes the kernels write into a plan's device error flag (0 = no error).
constexpr int kFlagNotSpd = 1;    // a Cholesky pivot was not positive / empty class
constexpr int kFlagDraw = 2;      // SRHT row draw left [0, n_pad)
constexpr int kFlagBucket = 3;    // CountSketch bucket index out of [0, s)
constexpr int kFlagTimeout = 4;   // a bounded device wait ran out (kernel aborted)
constexpr int kFlagLabel = 5;     // an FDA label outside [0, n_classes)

// Status and message for a flag value read back from the device.
inline int flag_status(int f) {
  switch (f) {
    case 0: return GBCCA_OK;
    case kFlagNotSpd:
      set_last_error("a Cholesky pivot was not positive (matrix not SPD)");
      return GBCCA_ERR_NOT_SPD;
    case kFlagBucket:
      set_last_error("CountSketch bucket index out of range");
      return GBCCA_ERR_INVALID_ARG;
    case kFlagLabel:
      set_last_error("a label is outside [0, n_classes)");
      return GBCCA_ERR_INVALID_ARG;
    case kFlagTimeout:
      set_last_error("a bounded device-side wait ran out; the kernel stopped early and its results are void");
      return GBCCA_ERR_TIMEOUT;
  }
  set_last_error("device-side check failed (flag " + std::to_string(f) + ")");
  return GBCCA_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- loads
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
// conversion to a kernel's working type T (FP32 work stays on FP32 units)
template <typename T> __device__ __forceinline__ T to_work(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T to_work(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T to_work(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

template <typename T> __device__ __forceinline__ T cvt(float v);
template <typename T> __device__ __forceinline__ T cvt(double v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cvt<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }

template <typename Tacc, typename Tin> __device__ __forceinline__ Tacc ld_as(const Tin* p);
template <> __device__ __forceinline__ float ld_as<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld_as<float, double>(const double* p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ double ld_as<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ double ld_as<double, float>(const float* p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ double ld_as<double, __nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(*p);
}

// ---------------------------------------------------------------- reductions
// 1/sqrt(x) for x > 0 in FP64: the single-precision estimate refined by two
// Newton-Raphson steps for f(y) = 1/y^2 - x, y <- y (3 - x y^2) / 2 (each
// step doubles the correct bits: ~2^-22 -> 2^-44 -> full precision).  Short
// dependent chains of FMAs instead of FP64 square root and division, which
// are long sequences on this GPU.  Outside the float range: 1 / sqrt(x).
__device__ __forceinline__ double rsqrt_nr(double x) {
  const float xf = (float)x;
  if (!(xf > 1e-37f && xf < 1e37f)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf(xf);
  const double hx = 0.5 * x;
  y = y * fma(-hx * y, y, 1.5);
  y = y * fma(-hx * y, y, 1.5);
  return y;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- SplitMix64
// Counter-based SplitMix64 (Steele, Lea & Flood 2014): the i-th output of the
// stream seeded with `seed`.
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kSaltSigns = 0xD1B54A32D192ED03ull;
constexpr uint64_t kSaltRows = 0x8CB92BA72F3D8DD7ull;

}  // namespace gbcca
