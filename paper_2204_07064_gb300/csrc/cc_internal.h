// Internal launch descriptors shared by the host runtime and the kernels.
//
// Every tensor edge of the reconfigured model lives, per stream, in a ring
// buffer of R rows x C channels (channels-last) inside the stream's arena
// slot.  Row r holds the frame whose absolute time index t satisfies
// t mod R == r.  A consumer that needs N frames of cached padding (section 2.2,
// Fig. 1) simply reads times t0 - N .. t0 - 1 from the ring: the "cache" is
// the previous call's tail, still in place, so no copy is ever made.  Rings
// start zeroed, which is the zero left padding of the causal model (section 3).
// A stream's absolute time at a node is (steps done) x (frames per step).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cc {

constexpr float kLeakySlope = 0.2f;

// Where one stream's frames of one node live.
struct Ring {
  int64_t off;   // byte offset inside a slot
  int32_t rows;  // R
  int32_t chans; // C
  int32_t u;     // frames per model step at this node
  int32_t dtype; // 0 f32, 1 bf16, 2 f16
};

// Streams of one launch: slot indices into the arena + per-slot counters.
struct Batch {
  char* arena;
  int64_t slot_bytes;
  const int32_t* slots;     // [count]
  const int64_t* counters;  // [max_streams] model steps done, by slot
  const uint64_t* seeds;    // [max_streams] noise seeds, by slot
  int32_t count;
};

// A convolution or transposed convolution as a GEMM over one launch:
//   D[M][N] = A[M][Kt] . B[N][Kt]^T,  N = count x ncols.
// Column j of stream s, reduction index (tap k, channel c):
//   B = act(in[time t0_in + j*stride + k*dil - hist][c]),  t0_in = steps*in.u
// Conv: row m is output channel m at time t0_out + j.
// ConvT (polyphase): row m = phase*cout + n is channel n at time
//   t0_out + j*phases + phase.
struct ConvArgs {
  const float* A;    // packed FP32 weights [M][Kt], Kt = taps*cin
  const float* bias; // [cout] or null
  int32_t M, Kt, taps, cin, dil, stride, hist, ncols, act;
  int32_t cout, phases; // phases = 1 for conv, S for convt
  Ring in, out;
  float* ext_out;       // if non-null the output goes here: stream s at
  int64_t ext_stride;   //   ext_out + s*ext_stride + local_time*cout + n
  int32_t has_skip;     // fused residual add: + skip[time - skip_A]
  int32_t skip_A;
  Ring skip;
  Batch batch;
};

struct HeadsArgs {
  Ring in[3];
  int32_t A[3];        // Eq. 3 alignment of each branch
  int64_t delay;       // cumulated delay at the heads (own frames): noise key offset
  int32_t bands, ncols, noise;
  Ring out;
  float* ext_out;
  int64_t ext_stride;
  Batch batch;
};

struct AddArgs {
  Ring in[2];
  int32_t A[2];
  int32_t ncols;
  Ring out;
  float* ext_out;
  int64_t ext_stride;
  Batch batch;
};

struct InputArgs {
  const float* src;   // count x [ncols][C]
  int64_t src_stride; // floats between streams
  int32_t ncols;
  Ring out;
  Batch batch;
};

// FP32 kernels (cc_kernels_f32.cu)
cudaError_t launch_conv_f32(const ConvArgs& a, cudaStream_t st);
cudaError_t launch_heads(const HeadsArgs& a, cudaStream_t st);
cudaError_t launch_add(const AddArgs& a, cudaStream_t st);
cudaError_t launch_input(const InputArgs& a, cudaStream_t st);
cudaError_t launch_advance(const Batch& b, int64_t steps, cudaStream_t st);

}  // namespace cc
