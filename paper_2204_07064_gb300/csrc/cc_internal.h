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
//
// A node's output may be kept in up to three views: FP32 as computed (read
// by residual merges, heads and FP32 layers) and low-precision copies with
// no activation or with LeakyReLU already applied (read by tensor-core
// layers, which stage them into shared memory unchanged).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace cc {

constexpr float kLeakySlope = 0.2f;

enum : int32_t { kDtF32 = 0, kDtBF16 = 1, kDtF16 = 2 };

// Where one stream's frames of one view of one node live.  rows == 0: absent.
// Frame t sits at ring row t mod R.  A low-precision view also keeps a copy
// of its last `pre` ring rows just before row 0 (rows -pre .. -1 mirror rows
// R-pre .. R-1, written together with them), so that a window of the cached
// history plus the frames of one call that starts in the ring's tail can be
// read as one run of consecutive rows.
struct Ring {
  int64_t off;    // byte offset inside a slot of ring row 0
  int32_t rows;   // R
  int32_t chans;  // C
  int32_t u;      // frames per model step at this node
  int32_t dtype;  // kDt*
  int32_t pre;    // mirrored rows before row 0 (low-precision views), else 0
  int32_t choff;  // first channel of this view inside the ring's rows (a sibling
                  // group's members share one ring of `chans` channels per row)
};

// Every destination of a layer's output.
struct OutViews {
  Ring f32;            // FP32 as computed
  Ring lp[2];          // low precision: [0] as computed, [1] LeakyReLU applied
  float* ext;          // caller's buffer (last node): stream s at ext + s*ext_stride
  int64_t ext_stride;  //   + local_time*C + channel
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
  const float* A;     // packed FP32 weights [M][Kt], Kt = taps*cin
  const float* bias;  // [cout] or null
  int32_t M, Kt, taps, cin, dil, stride, hist, ncols, act;
  int32_t cout, phases;  // phases = 1 for conv, S for convt
  int32_t out_u;         // output frames per step
  Ring in;               // FP32 view of the input
  OutViews out;
  int32_t has_skip;  // fused residual add: + skip[time - skip_A] (FP32 view)
  int32_t skip_A;
  Ring skip;
  Batch batch;
  int32_t advance;  // last launch of a chain: add this many steps to the streams' counters
};

// Tensor-core form of ConvArgs: A is low precision [Mpad][Kt] stored as
// pre-swizzled 128 x 64 blocks, row m scaled by scale[m]; B is read from the
// input's low-precision view (activation pre-applied).
struct TcArgs {
  const void* A_tiled;  // weights as [Mpad/128][Kt/64] blocks of 128 x 64, each 16 KB in the
                        // 128-byte-swizzled K-major order (one bulk copy per block)
  const float* scale;   // [Mpad]
  const float* bias;   // [cout] or null
  int32_t M, Kt, taps, cin, dil, stride, hist, ncols, cout, phases, out_u;
  Ring in;
  int32_t in_rows_per_slot;  // the input view seen as rows of the whole arena:
  int32_t in_row_off;        //   row = slot*in_rows_per_slot + in_row_off + ring row
  int32_t box_ok;            // stride 1 and ncols divides 128 or is a multiple of it:
                             //   tiles of consecutive slots at one step may load their
                             //   window rows as 3D boxes (tmap_t) instead of gathers
  OutViews out;
  int32_t has_skip, skip_A;
  int32_t skip_early;  // the residual's producer launched two or more launches back
  int32_t ksplit;      // split-K factor (1, 2 or 4): CTAs per cluster sharing a tile
  int32_t deep_ok;     // one-wave grids may take the deep one-CTA-per-SM pipelines (models
                       //   sized for at most 256 streams: no concurrent chains expected)
  int32_t mdup;        // M <= 64 and the weight tiles (A and A2) repeat rows 0..63 in rows
                       //   64..127: accumulator lanes 64..127 repeat lanes 0..63, so all
                       //   four TMEM lane quarters have rows to store (split the columns)
  // Residual-unit fusion (k2 > 0): the tile's result, scaled, biased and
  // activated (act2) in BF16/FP16, is the B operand of a second, 1x1
  // contraction A2 [M][k2*64] (pre-tiled like A) whose result, with scale2,
  // bias2, the residual and the views above, is the launch's output.
  const void* A2_tiled;
  const float* scale2;
  const float* bias2;
  int32_t k2, act2;
  Ring skip;
  Batch batch;
  int32_t* err;      // device error word: set when a bounded wait gives up
  uint64_t wait_ns;  // limit of every pipeline wait
  int32_t* withhold;  // failure-detection test counter (see the producer)
};

struct HeadsArgs {
  Ring in[3];
  int32_t A[3];   // Eq. 3 alignment of each branch
  int64_t delay;  // cumulated delay at the heads (own frames): noise key offset
  int32_t bands, ncols, noise, out_u;
  OutViews out;
  Batch batch;
};

struct AddArgs {
  Ring in[2];
  int32_t A[2];
  int32_t ncols, chans, out_u;
  OutViews out;
  Batch batch;
};

struct InputArgs {
  const float* src;     // count x [ncols][C]
  int64_t src_stride;   // floats between streams
  const float* manip;   // [max_streams][3][C] by slot: scale, bias, noise-amplitude rows
  int32_t ncols, chans, out_u;
  OutViews out;
  Batch batch;
};

// Launch with programmatic stream serialization (see pdl_wait / pdl_release):
// the kernel's prologue may overlap the previous kernel of the stream.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// FP32 kernels (cc_kernels_f32.cu)
cudaError_t launch_conv_f32(const ConvArgs& a, cudaStream_t st);
// The narrow FP32 kernel can advance the step counters itself (ConvArgs.advance)
// when each of its 128-column blocks covers whole streams.
bool conv_f32_can_advance(const ConvArgs& a);
cudaError_t launch_heads(const HeadsArgs& a, cudaStream_t st);
cudaError_t launch_add(const AddArgs& a, cudaStream_t st);
cudaError_t launch_input(const InputArgs& a, cudaStream_t st);
cudaError_t launch_advance(const Batch& b, int64_t steps, cudaStream_t st);

// Tensor-core kernels (cc_kernels_tc.cu).  tmap_t: the input view as
// [slot][pre + R rows][C], boxes of 64 channels x min(ncols, 128) rows x
// 128 / that many slots; tmap_b: the input view as arena rows of C elements,
// one-row boxes of 64 (gathered four rows at a time).  Both CUtensorMap (128 B).
cudaError_t launch_conv_tc(const void* tmap_t, const void* tmap_b, const TcArgs& a, int bn,
                           cudaStream_t st);
int tc_tile_n(int64_t n_cols, int m_tiles);

}  // namespace cc
