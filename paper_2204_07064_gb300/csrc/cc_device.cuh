// Device helpers shared by the kernels: ring addressing, activation, the
// multi-view output store and the counter-based noise.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cc_internal.h"

namespace cc {

__device__ __forceinline__ int64_t ring_row(int64_t t, int32_t rows) {
  int64_t r = t % rows;
  return r < 0 ? r + rows : r;
}

__device__ __forceinline__ int32_t wrap_row(int32_t r, int32_t rows) {
  return r >= rows ? r - rows : r;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is still
// running.  pdl_wait() blocks until the predecessor grid has completed and its
// memory is visible; everything before it may only touch data no earlier
// kernel of the chain writes (weights, tensor maps, shared memory, TMEM).
// pdl_release() lets the next kernel start launching; it is issued only after
// pdl_wait(), so a kernel never overlaps a kernel two places earlier.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float leaky(float x) { return x < 0.f ? kLeakySlope * x : x; }

__device__ __forceinline__ float activate(float x, int32_t act) { return act ? leaky(x) : x; }

__device__ __forceinline__ char* slot_base(const Batch& b, int32_t s) {
  return b.arena + (int64_t)b.slots[s] * b.slot_bytes;
}

template <typename T>
__device__ __forceinline__ T* ring_ptr(const Batch& b, int32_t s, const Ring& r) {
  return reinterpret_cast<T*>(slot_base(b, s) + r.off);
}

__device__ __forceinline__ int64_t steps_of(const Batch& b, int32_t s) {
  return b.counters[b.slots[s]];
}

// Low-precision store of ring row `row` (0 <= row < R), and of its mirror
// row - R when the row lies in the ring's mirrored tail.
__device__ __forceinline__ void store_lp(char* base, const Ring& r, int64_t row, int32_t ch, float x) {
  const bool mirror = row >= r.rows - r.pre;
  if (r.dtype == kDtBF16) {
    __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base + r.off);
    const __nv_bfloat16 v = __float2bfloat16_rn(x);
    p[row * r.chans + ch] = v;
    if (mirror) p[(row - r.rows) * r.chans + ch] = v;
  } else {
    __half* p = reinterpret_cast<__half*>(base + r.off);
    const __half v = __float2half_rn(x);
    p[row * r.chans + ch] = v;
    if (mirror) p[(row - r.rows) * r.chans + ch] = v;
  }
}

// Writes value v of channel ch at absolute time t (local time lt within this
// call) of stream s into every view of `o`.
__device__ __forceinline__ void store_views(const Batch& b, int32_t s, const OutViews& o, int64_t t,
                                            int32_t lt, int32_t ch, int32_t chans, float v) {
  char* base = slot_base(b, s);
  if (o.ext) o.ext[(int64_t)s * o.ext_stride + (int64_t)lt * chans + ch] = v;
  if (o.f32.rows)
    reinterpret_cast<float*>(base + o.f32.off)[ring_row(t, o.f32.rows) * o.f32.chans + ch] = v;
  if (o.lp[0].rows) store_lp(base, o.lp[0], ring_row(t, o.lp[0].rows), ch, v);
  if (o.lp[1].rows) store_lp(base, o.lp[1], ring_row(t, o.lp[1].rows), ch, leaky(v));
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator: its
// (n+1)-th output from `seed` is mix(seed + (n+1) * 0x9E3779B97F4A7C15), so
// any (stream, band, frame) draws its value directly.
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// u in [-1, 1) (exact in float32) for band `band` of `bands` at frame
// `frame`: counter = frame * bands + band.
__device__ __forceinline__ float noise_uniform(uint64_t seed, int64_t frame, int32_t band, int32_t bands) {
  const uint64_t counter = (uint64_t)(frame * bands + band);
  const uint64_t z = splitmix_mix(seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
  return (float)(z >> 40) * 0x1p-23f - 1.0f;
}

}  // namespace cc
