// Backward pass of the streamed (causally reconfigured) model, one chunk at a
// time, in reverse time order.
//
// The streamed output equals the causal offline model (section 4.2), so the
// gradient of a loss over a long streamed signal is that model's gradient.
// It is computed chunk by chunk, last chunk first, with per-chunk activation
// checkpointing: the caller restores the stream state saved at the chunk's
// start, the chunk's forward is recomputed (the rings then hold every
// activation the chunk read or wrote, history included), and the adjoints
// are propagated backwards through the nodes.
//
// Adjoints live in an "adjoint arena" with the same slot layout as the FP32
// views of the forward rings, indexed by the same absolute times.  A layer
// that read N cached frames (section 2.2) scatters their adjoint into times
// t0-N .. t0-1 of its input's adjoint ring; those rows are left in place and
// are exactly the cache adjoint the previous chunk starts from.  Before a
// chunk, only the rows that no later chunk could have touched are cleared.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/cachedconv.h"
#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {
int32_t stream_slot(const cc_stream* s);
bool stream_manipulated(const cc_stream* s);
Model* stream_model(const cc_stream* s);
}  // namespace cc

namespace {

using namespace cc;

// Forward values a backward kernel reads: the view the forward computed with.
// kind 0: FP32 pre-activation values (the consumer's activation is applied on
// read); 1: low precision as computed; 2: low precision with LeakyReLU
// applied (what a tensor-core layer multiplied; its sign is the pre-activation's).
struct ValView {
  Ring r;
  int32_t kind, act, lp_bf16;
};

__device__ __forceinline__ float load_lp(const void* p, bool bf16) {
  const uint16_t h = *reinterpret_cast<const uint16_t*>(p);
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// Start of the row the forward wrote at time t (FP32 views: at the node's
// channel offset; low-precision views: 2 bytes per channel).
__device__ __forceinline__ const char* val_row(const Batch& b, int32_t s, const ValView& v, int64_t t) {
  const char* base = slot_base(b, s) + v.r.off;
  const int64_t row = ring_row(t, v.r.rows);
  return v.kind == 0 ? base + (row * v.r.chans + v.r.choff) * 4 : base + row * v.r.chans * 2;
}

// The value the forward multiplied (activation applied), channel m of a row.
__device__ __forceinline__ float val_at(const char* row, const ValView& v, int32_t m) {
  if (v.kind == 0) return activate(reinterpret_cast<const float*>(row)[m], v.act);
  return load_lp(row + m * 2, v.lp_bf16 != 0);
}

// The activation's derivative there (1 without activation).
__device__ __forceinline__ float deriv_at(const char* row, const ValView& v, int32_t m) {
  if (v.kind == 1 || (v.kind == 0 && !v.act)) return 1.f;
  return val_at(row, v, m) >= 0.f ? 1.f : kLeakySlope;  // LeakyReLU keeps the sign
}

// Adjoint rows: an FP32 ring per node in the adjoint arena, indexed by the
// node's absolute time like the forward rings.
__device__ __forceinline__ float* adj_row(char* adj, int64_t adj_slot_bytes, int32_t slot, const Ring& r, int64_t t) {
  return reinterpret_cast<float*>(adj + (int64_t)slot * adj_slot_bytes + r.off) + ring_row(t, r.rows) * r.chans;
}

__device__ __forceinline__ int64_t chunk_t0(const Batch& b, int32_t s, int32_t u, int32_t steps) {
  return (steps_of(b, s) - steps) * (int64_t)u;
}

// Zero the adjoint rows of times [t0 - keep, t0 + n - keep) for every stream
// and every listed ring: the rows no later chunk (processed earlier, in
// reverse order) could have written; rows [t0 + n - keep, t0 + n) hold the
// cache adjoint they left.  One launch covers up to kClearMax rings; entry k
// owns elements [start[k], start[k + 1]) of the flattened (stream, row,
// channel) space.
constexpr int kClearMax = 48;
struct ClearList {
  int32_t count;
  Ring r[kClearMax];
  int32_t keep[kClearMax], n[kClearMax];
  int64_t start[kClearMax + 1];
};

__global__ void k_adj_clear(Batch b, char* adj, int64_t adj_slot_bytes, const __grid_constant__ ClearList L,
                            int32_t steps) {
  const int64_t total = L.start[L.count];
  int32_t k = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    while (i >= L.start[k + 1]) ++k;  // i only grows within a thread
    const Ring& r = L.r[k];
    const int64_t e = i - L.start[k];
    const int32_t c = (int32_t)(e % r.chans);
    const int64_t q = e / r.chans;
    const int32_t j = (int32_t)(q % L.n[k]);
    const int32_t s = (int32_t)(q / L.n[k]);
    const int64_t t = chunk_t0(b, s, r.u, steps) - L.keep[k] + j;
    adj_row(adj, adj_slot_bytes, b.slots[s], r, t)[c] = 0.f;
  }
}

struct BwdConv {
  const float* Wt;  // weights per tap: [K][cout][cin] (what the forward multiplied)
  int32_t op;       // CC_OP_CONV / CC_OP_CONVT
  int32_t cin, cout, K, S, dil, hist;
  int32_t n_in, n_out;  // frames of this chunk per stream, input / output rate
  ValView x;            // the forward's input values
  int32_t u_in, u_out;
  Ring gy;              // adjoint ring of the output node (rows == 0: gy_ext)
  const float* gy_ext;  // caller's output gradient, stream s at gy_ext + s*gy_stride
  int64_t gy_stride;
  Ring gx;              // adjoint ring of the input node
  float* dW;            // accumulators, tap-major [K][cout][cin]
  float* db;
  int32_t steps;
  Batch b;
  char* adj;
  int64_t adj_slot_bytes;
  // split reductions: blockIdx.z = (tap or 0) * splits + split; with splits >
  // 1 every split writes a 64 x 64 partial of its tile and the tile's last
  // block to arrive adds them, in split order, into the destination
  int32_t splits;
  int32_t res;         // dX rows residue by residue (strided convolution, dilation 1)
  int64_t per_split;   // reduction steps per split: columns (dW), (tap, 32-channel chunk) pairs (dX)
  float* part;         // [tile][split][64 * 64]
  float* bpart;        // [n tile][phase][split][64] bias partials (dW)
  uint32_t* counters;  // per tile arrivals, then per n tile bias arrivals; left at 0
};

__device__ __forceinline__ const float* gy_row(const BwdConv& a, int32_t s, int64_t t_local, int64_t t0_out) {
  if (a.gy.rows == 0) return a.gy_ext + (int64_t)s * a.gy_stride + t_local * a.cout;
  return adj_row(a.adj, a.adj_slot_bytes, a.b.slots[s], a.gy, t0_out + t_local);
}

constexpr int kBT = 64;  // output tile (rows x columns) of the backward GEMMs
constexpr int kBC = 32;  // reduction chunk
// split reductions aim at 4 blocks per SM; the partial buffer holds twice
// that many 64 x 64 tiles, and the bias arrival counters sit after the tiles'
constexpr int64_t kTargetBlocks = 4 * 152;
constexpr int64_t kPartTiles = 2 * kTargetBlocks;

// Split reductions: a block's 4 x 4 accumulators (rows ty*4+i, columns
// tx*4+j of its 64 x 64 tile) go straight to `apply` when the reduction is not
// split; otherwise into the tile's partial for this split, and the last split
// to arrive sums the tile's partials in split order (deterministic) and
// applies the sum.  Returns whether this block applied the tile.
template <typename Apply>
__device__ __forceinline__ bool finish_tile(const BwdConv& a, float (&acc)[4][4], int64_t tile, int32_t split,
                                            Apply apply) {
  const int32_t tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (a.splits == 1) {
    apply(acc);
    return true;
  }
  __shared__ bool last;
  float* mine = a.part + (tile * a.splits + split) * (kBT * kBT);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(mine + (ty * 4 + i) * kBT + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t prev = atomicAdd(a.counters + tile, 1u);
    last = prev == (uint32_t)a.splits - 1;
    if (last) a.counters[tile] = 0;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  float sum[4][4] = {};
#pragma unroll 4
  for (int32_t q = 0; q < a.splits; ++q) {
    const float* p = a.part + (tile * a.splits + q) * (kBT * kBT);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p + (ty * 4 + i) * kBT + tx * 4));
      sum[i][0] += v.x;
      sum[i][1] += v.y;
      sum[i][2] += v.z;
      sum[i][3] += v.w;
    }
  }
  apply(sum);
  return true;
}

// dL/dW of this chunk as a GEMM per tap k: dW_k[n][m] += sum over columns
// (stream, output frame) of gy[col][n] * x_k[col][m], x_k the value the
// forward multiplied by tap k.  A block computes a 64 x 64 tile of one tap
// over one split of the columns; 4 x 4 outputs per thread.  (A transposed
// convolution's tap kk = ph + jj*S pairs output phase ph with input frame
// q - jj.)  dL/db, the sum of gy over every output frame, rides along in the
// blocks of the first input-channel tile: tap 0 of a convolution, taps
// 0..S-1 (one per output phase) of a transposed one; with more than one such
// block per output-channel tile, the last to arrive sums their partials in
// (phase, split) order.
__global__ void __launch_bounds__(256) k_bwd_weight(BwdConv a) {
  __shared__ __align__(16) float Gs[kBC][kBT + 4];
  __shared__ __align__(16) float Xs[kBC][kBT + 4];
  __shared__ const float* gp[2][kBC];  // row pointers of a chunk's columns, two chunks in flight
  __shared__ const char* xp[2][kBC];
  __shared__ bool blast;
  const int32_t n0 = blockIdx.x * kBT, m0 = blockIdx.y * kBT;
  const int32_t kk = blockIdx.z / a.splits, split = blockIdx.z - kk * a.splits;
  const int32_t tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool convt = a.op == CC_OP_CONVT;
  const int32_t ph = convt ? kk % a.S : 0, jj = convt ? kk / a.S : 0;
  const int32_t ncol = convt ? a.n_in : a.n_out;
  const int64_t total = (int64_t)a.b.count * ncol;
  const int64_t c_begin = (int64_t)split * a.per_split;
  const int64_t c_end = c_begin + a.per_split < total ? c_begin + a.per_split : total;
  const bool bias = a.db && blockIdx.y == 0 && (convt ? kk < a.S : kk == 0);
  const int32_t nph = convt ? a.S : 1;
  float acc[4][4] = {};
  float bacc = 0.f;
  // Software pipeline over chunks of kBC columns: the row pointers of chunk
  // i + 2 are computed, and chunk i + 1's values are loaded into registers,
  // while chunk i is multiplied out of shared memory.
  auto set_ptrs = [&](int64_t c0, int b) {
    if (threadIdx.x < kBC) {
      const int64_t col = c0 + threadIdx.x;
      const float* g = nullptr;
      const char* xr = nullptr;
      if (col < c_end) {
        const int32_t s = (int32_t)(col / ncol), o = (int32_t)(col - (int64_t)s * ncol);
        const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
        g = gy_row(a, s, convt ? (int64_t)o * a.S + ph : o, t0_out);
        xr = val_row(a.b, s, a.x, convt ? t0_in + o - jj : t0_in + (int64_t)o * a.S + (int64_t)kk * a.dil - a.hist);
      }
      gp[b][threadIdx.x] = g;
      xp[b][threadIdx.x] = xr;
    }
  };
  constexpr int kPer = kBC * kBT / 256;  // elements per thread per chunk
  float rg[kPer], rx[kPer];
  auto load = [&](int b) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int e = threadIdx.x + 256 * r, c = e / kBT, q = e - c * kBT;
      float g = 0.f, x = 0.f;
      const float* gr = gp[b][c];
      if (gr) {
        if (n0 + q < a.cout) g = gr[n0 + q];
        if (m0 + q < a.cin) x = val_at(xp[b][c], a.x, m0 + q);
      }
      rg[r] = g;
      rx[r] = x;
    }
  };
  set_ptrs(c_begin, 0);
  set_ptrs(c_begin + kBC, 1);
  __syncthreads();
  load(0);
  int cur = 0;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kBC, cur ^= 1) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int e = threadIdx.x + 256 * r, c = e / kBT, q = e - c * kBT;
      Gs[c][q] = rg[r];
      Xs[c][q] = rx[r];
    }
    __syncthreads();  // the chunk's tile is complete; chunk i + 1's pointers are visible
    if (c0 + kBC < c_end) load(cur ^ 1);
    set_ptrs(c0 + 2 * kBC, cur);  // (this buffer's loads were issued a chunk ago)
    if (bias && threadIdx.x < kBT)
      for (int c = 0; c < kBC; ++c) bacc += Gs[c][threadIdx.x];
#pragma unroll 4
    for (int c = 0; c < kBC; ++c) {
      const float4 g4 = *reinterpret_cast<const float4*>(&Gs[c][ty * 4]);
      const float4 x4 = *reinterpret_cast<const float4*>(&Xs[c][tx * 4]);
      const float g[4] = {g4.x, g4.y, g4.z, g4.w}, x[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) acc[i][j2] = fmaf(g[i], x[j2], acc[i][j2]);
    }
    __syncthreads();
  }
  const int64_t tile = ((int64_t)kk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  // dW accumulates tap-major, [K][cout][cin] like Wt: a thread's 4 input
  // channels are one 16-byte word when cin allows
  const bool vec = (a.cin & 3) == 0;
  finish_tile(a, acc, tile, split, [&](float (&v)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int32_t n = n0 + ty * 4 + i, m = m0 + tx * 4;
      if (n >= a.cout || m >= a.cin) continue;
      float* w = a.dW + ((int64_t)kk * a.cout + n) * a.cin + m;
      if (vec) {
        float4 t = *reinterpret_cast<float4*>(w);
        t.x += v[i][0];
        t.y += v[i][1];
        t.z += v[i][2];
        t.w += v[i][3];
        *reinterpret_cast<float4*>(w) = t;
      } else {
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2)
          if (m + j2 < a.cin) w[j2] += v[i][j2];
      }
    }
  });
  if (!bias) return;
  const int32_t contributors = nph * a.splits;
  if (contributors == 1) {
    if (threadIdx.x < kBT && n0 + (int32_t)threadIdx.x < a.cout) a.db[n0 + threadIdx.x] += bacc;
    return;
  }
  if (threadIdx.x < kBT) a.bpart[(((int64_t)blockIdx.x * nph + ph) * a.splits + split) * kBT + threadIdx.x] = bacc;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t* cnt = a.counters + kPartTiles + blockIdx.x;
    const uint32_t prev = atomicAdd(cnt, 1u);
    blast = prev == (uint32_t)contributors - 1;
    if (blast) *cnt = 0;
  }
  __syncthreads();
  if (!blast) return;
  __threadfence();
  if (threadIdx.x < kBT && n0 + (int32_t)threadIdx.x < a.cout) {
    float sb = 0.f;
    for (int32_t q = 0; q < contributors; ++q)
      sb += __ldcg(a.bpart + ((int64_t)blockIdx.x * contributors + q) * kBT + threadIdx.x);
    a.db[n0 + threadIdx.x] += sb;
  }
}

// dL/dx for the chunk's input frames i in [-hist, n_in) (the cached history
// included), times the activation's derivative, added into the input's
// adjoint ring: a GEMM over (tap, output channel) per (stream, frame) row,
// the (tap, 32-channel chunk) steps of the reduction split across
// blockIdx.z.  Only this chunk's output frames contribute; later chunks
// already added theirs into these rows.  For a strided convolution of
// dilation 1 (a.res) the rows are taken residue by residue: frame e = i +
// hist only meets taps k = e mod S + S*jt, so a block holds rows of one
// residue and runs only those ceil(K/S) taps.
__global__ void __launch_bounds__(256) k_bwd_data(BwdConv a) {
  __shared__ __align__(16) float Gs[kBC][kBT + 4];  // [n][row]
  __shared__ __align__(16) float Ws[kBC][kBT + 4];  // [n][m]
  __shared__ const float* gp[2][kBT];  // gy row of each tile row for a step's tap, two steps in flight
  __shared__ int32_t rs[kBT];
  __shared__ int32_t ri[kBT];
  const int32_t span = a.hist + a.n_in;
  const int64_t rows = (int64_t)a.b.count * span;
  const int64_t r0 = (int64_t)blockIdx.x * kBT;
  const int32_t m0 = blockIdx.y * kBT;
  const int32_t split = blockIdx.z;
  const int32_t tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool convt = a.op == CC_OP_CONVT;
  // residue mode: this block's residue and its first row within it
  int32_t res = 0, nj = span;
  int64_t rbase = r0;
  if (a.res) {
    int64_t bx = blockIdx.x;
    for (res = 0; res < a.S; ++res) {
      nj = (span - res + a.S - 1) / a.S;
      const int64_t t = ((int64_t)a.b.count * nj + kBT - 1) / kBT;
      if (bx < t) break;
      bx -= t;
    }
    rbase = bx * kBT;
  }
  if (threadIdx.x < kBT) {
    const int64_t row = rbase + threadIdx.x;
    rs[threadIdx.x] = -1;
    ri[threadIdx.x] = 0;
    if (a.res) {
      if (row < (int64_t)a.b.count * nj) {
        rs[threadIdx.x] = (int32_t)(row / nj);
        ri[threadIdx.x] = res + a.S * (int32_t)(row - (int64_t)rs[threadIdx.x] * nj) - a.hist;
      }
    } else if (row < rows) {
      rs[threadIdx.x] = (int32_t)(row / span);
      ri[threadIdx.x] = (int32_t)(row - (int64_t)rs[threadIdx.x] * span) - a.hist;
    }
  }
  const int32_t nch = (a.cout + kBC - 1) / kBC;
  const int32_t ntaps = a.res ? (a.K > res ? (a.K - res + a.S - 1) / a.S : 0) : a.K;
  const int64_t steps_total = (int64_t)ntaps * nch;
  const int64_t it_begin = (int64_t)split * a.per_split;
  const int64_t it_end = it_begin + a.per_split < steps_total ? it_begin + a.per_split : steps_total;
  float acc[4][4] = {};
  // Software pipeline over the (tap, 32-channel chunk) steps: the gy rows of
  // step i + 2's tap are found, and step i + 1's gy and W values are loaded
  // into registers, while step i is multiplied out of shared memory.
  auto tap_of = [&](int64_t it) -> int32_t {
    const int32_t jt = (int32_t)(it / nch);
    return a.res ? res + a.S * jt : jt;
  };
  auto set_gp = [&](int64_t it, int b) {
    if (threadIdx.x < kBT) {
      const int32_t s = rs[threadIdx.x], i = ri[threadIdx.x];
      const float* p = nullptr;
      if (s >= 0 && it < it_end) {
        const int32_t tap = tap_of(it);
        const int64_t t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
        if (!convt) {
          const int32_t jj2 = i + a.hist - tap * a.dil;
          if (jj2 >= 0 && jj2 % a.S == 0 && jj2 / a.S < a.n_out) p = gy_row(a, s, jj2 / a.S, t0_out);
        } else {
          const int32_t ph = tap % a.S, jj = tap / a.S, qq = i + jj;
          if (qq >= 0 && qq < a.n_in) p = gy_row(a, s, (int64_t)qq * a.S + ph, t0_out);
        }
      }
      gp[b][threadIdx.x] = p;
    }
  };
  constexpr int kPer = kBC * kBT / 256;  // elements of each operand per thread per step
  float rg[kPer], rw[kPer];
  auto load = [&](int64_t it, int b) {
    const int32_t tap = tap_of(it), n0 = (int32_t)(it - (int64_t)(it / nch) * nch) * kBC;
    const float* wt = a.Wt + (int64_t)tap * a.cout * a.cin;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int e = threadIdx.x + 256 * r;
      {  // gy: a warp reads 32 consecutive channels of one row (coalesced)
        const int q = e / kBC, c = e - q * kBC;
        const int32_t n = n0 + c;
        const float* g = gp[b][q];
        rg[r] = (g && n < a.cout) ? g[n] : 0.f;
      }
      {  // W: a warp reads along input channels
        const int c = e / kBT, q = e - c * kBT;
        const int32_t n = n0 + c;
        rw[r] = (n < a.cout && m0 + q < a.cin) ? wt[(int64_t)n * a.cin + m0 + q] : 0.f;
      }
    }
  };
  set_gp(it_begin, 0);
  set_gp(it_begin + 1, 1);
  __syncthreads();
  if (it_begin < it_end) load(it_begin, 0);
  int cur = 0;
  for (int64_t it = it_begin; it < it_end; ++it, cur ^= 1) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int e = threadIdx.x + 256 * r;
      {
        const int q = e / kBC, c = e - q * kBC;
        Gs[c][q] = rg[r];
      }
      {
        const int c = e / kBT, q = e - c * kBT;
        Ws[c][q] = rw[r];
      }
    }
    __syncthreads();  // the step's tiles are complete; step i + 1's gy rows are visible
    if (it + 1 < it_end) load(it + 1, cur ^ 1);
    set_gp(it + 2, cur);  // (this buffer's loads were issued a step ago)
#pragma unroll 4
    for (int c = 0; c < kBC; ++c) {
      const float4 g4 = *reinterpret_cast<const float4*>(&Gs[c][ty * 4]);
      const float4 w4 = *reinterpret_cast<const float4*>(&Ws[c][tx * 4]);
      const float g[4] = {g4.x, g4.y, g4.z, g4.w}, w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
      for (int i2 = 0; i2 < 4; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) acc[i2][j2] = fmaf(g[i2], w[j2], acc[i2][j2]);
    }
    __syncthreads();
  }
  const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  finish_tile(a, acc, tile, split, [&](float (&v)[4][4]) {
#pragma unroll
    for (int i2 = 0; i2 < 4; ++i2) {
      const int32_t lr = ty * 4 + i2;
      const int32_t s = rs[lr];
      if (s < 0) continue;
      const int64_t t = chunk_t0(a.b, s, a.u_in, a.steps) + ri[lr];
      float* out = adj_row(a.adj, a.adj_slot_bytes, a.b.slots[s], a.gx, t);
      const char* xr = val_row(a.b, s, a.x, t);
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) {
        const int32_t m = m0 + tx * 4 + j2;
        if (m >= a.cin) continue;
        out[m] += v[i2][j2] * deriv_at(xr, a.x, m);
      }
    }
  });
}

// Layers with fewer than 16 input or output channels (the PQMF filterbanks)
// would leave most of a 64 x 64 tile idle; their gradients are a few million
// multiply-adds, computed directly.

// dL/dW (and dL/db) of a narrow layer: one block per weight (tap-major index
// ((kk * cout + n) * cin + m)), its threads striding over the columns, summed
// in a fixed order.
__global__ void __launch_bounds__(256) k_bwd_weight_narrow(BwdConv a) {
  __shared__ float red[2][8];
  const int64_t o = blockIdx.x;
  const int32_t m = (int32_t)(o % a.cin);
  const int64_t r = o / a.cin;
  const int32_t n = (int32_t)(r % a.cout), kk = (int32_t)(r / a.cout);
  const bool convt = a.op == CC_OP_CONVT;
  const int32_t ph = convt ? kk % a.S : 0, jj = convt ? kk / a.S : 0;
  const int32_t ncol = convt ? a.n_in : a.n_out;
  const int64_t total = (int64_t)a.b.count * ncol;
  const bool bias = a.db && m == 0 && kk == 0;
  float acc = 0.f, bacc = 0.f;
  for (int64_t col = threadIdx.x; col < total; col += blockDim.x) {
    const int32_t s = (int32_t)(col / ncol), q = (int32_t)(col - (int64_t)s * ncol);
    const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
    const float g = gy_row(a, s, convt ? (int64_t)q * a.S + ph : q, t0_out)[n];
    const int64_t t = convt ? t0_in + q - jj : t0_in + (int64_t)q * a.S + (int64_t)kk * a.dil - a.hist;
    acc = fmaf(g, val_at(val_row(a.b, s, a.x, t), a.x, m), acc);
    if (bias) {
      if (!convt) {
        bacc += g;
      } else {
        for (int32_t p = 0; p < a.S; ++p) bacc += gy_row(a, s, (int64_t)q * a.S + p, t0_out)[n];
      }
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, d);
    bacc += __shfl_xor_sync(0xffffffffu, bacc, d);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = acc;
    red[1][w] = bacc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float sw = 0.f, sb = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sw += red[0][k];
      sb += red[1][k];
    }
    a.dW[o] += sw;
    if (bias) a.db[n] += sb;
  }
}

// dL/dx of a narrow layer: one thread per (stream, frame, input channel),
// history frames included, summing its taps' output channels directly.
__global__ void __launch_bounds__(256) k_bwd_data_narrow(BwdConv a) {
  const int32_t span = a.hist + a.n_in;
  const int64_t total = (int64_t)a.b.count * span * a.cin;
  const bool convt = a.op == CC_OP_CONVT;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = (int32_t)(idx % a.cin);
    const int64_t row = idx / a.cin;
    const int32_t s = (int32_t)(row / span), i = (int32_t)(row - (int64_t)s * span) - a.hist;
    const int64_t t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
    float acc = 0.f;
    // a stride-S convolution of dilation 1 meets this frame with taps
    // k = (i + hist) mod S + S*j only
    const bool res = !convt && a.S > 1 && a.dil == 1;
    const int32_t tap0 = res ? (i + a.hist) % a.S : 0, tstep = res ? a.S : 1;
    for (int32_t tap = tap0; tap < a.K; tap += tstep) {
      const float* g = nullptr;
      if (!convt) {
        const int32_t jj2 = i + a.hist - tap * a.dil;
        if (jj2 >= 0 && jj2 % a.S == 0 && jj2 / a.S < a.n_out) g = gy_row(a, s, jj2 / a.S, t0_out);
      } else {
        const int32_t ph = tap % a.S, jj = tap / a.S, qq = i + jj;
        if (qq >= 0 && qq < a.n_in) g = gy_row(a, s, (int64_t)qq * a.S + ph, t0_out);
      }
      if (!g) continue;
      const float* w = a.Wt + (int64_t)tap * a.cout * a.cin + m;
      for (int32_t n = 0; n < a.cout; ++n) acc = fmaf(g[n], w[(int64_t)n * a.cin], acc);
    }
    const int64_t t = chunk_t0(a.b, s, a.u_in, a.steps) + i;
    adj_row(a.adj, a.adj_slot_bytes, a.b.slots[s], a.gx, t)[m] += acc * deriv_at(val_row(a.b, s, a.x, t), a.x, m);
  }
}

// dL/dW (and dL/db) of a narrow layer whose taps hold at most NW weights
// (cout x cin; both PQMF filterbanks have 16): blocks over (tap, split of the
// columns), each thread accumulating every weight of the tap over its
// columns, so a column's rows are found once.  A block's sums are reduced in
// a fixed order; with several splits the tap's last block to arrive adds the
// splits' partials in split order.
template <int NW>
__global__ void __launch_bounds__(256) k_bwd_weight_tap(BwdConv a) {
  __shared__ float red[2][8][NW + 1];
  __shared__ float tot[2][NW];
  __shared__ bool last;
  const int32_t kk = blockIdx.x, split = blockIdx.y;
  const bool convt = a.op == CC_OP_CONVT;
  const int32_t ph = convt ? kk % a.S : 0, jj = convt ? kk / a.S : 0;
  const int32_t ncol = convt ? a.n_in : a.n_out;
  const int64_t total = (int64_t)a.b.count * ncol;
  const int64_t c_begin = (int64_t)split * a.per_split;
  const int64_t c_end = c_begin + a.per_split < total ? c_begin + a.per_split : total;
  const int32_t nw = a.cout * a.cin;
  const bool bias = a.db && kk == 0;
  float acc[NW], bacc[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) acc[j] = bacc[j] = 0.f;
  for (int64_t col = c_begin + threadIdx.x; col < c_end; col += blockDim.x) {
    const int32_t s = (int32_t)(col / ncol), q = (int32_t)(col - (int64_t)s * ncol);
    const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
    const float* g = gy_row(a, s, convt ? (int64_t)q * a.S + ph : q, t0_out);
    const int64_t t = convt ? t0_in + q - jj : t0_in + (int64_t)q * a.S + (int64_t)kk * a.dil - a.hist;
    const char* xr = val_row(a.b, s, a.x, t);
#pragma unroll
    for (int j = 0; j < NW; ++j)
      if (j < nw) acc[j] = fmaf(g[j / a.cin], val_at(xr, a.x, j % a.cin), acc[j]);
    if (bias) {
      if (!convt) {
#pragma unroll
        for (int j = 0; j < NW; ++j)
          if (j < a.cout) bacc[j] += g[j];
      } else {
        for (int32_t p = 0; p < a.S; ++p) {
          const float* gp = gy_row(a, s, (int64_t)q * a.S + p, t0_out);
#pragma unroll
          for (int j = 0; j < NW; ++j)
            if (j < a.cout) bacc[j] += gp[j];
        }
      }
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    float x = acc[j], y = bacc[j];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, d);
      y += __shfl_xor_sync(0xffffffffu, y, d);
    }
    if (lane == 0) {
      red[0][w][j] = x;
      red[1][w][j] = y;
    }
  }
  __syncthreads();
  if (threadIdx.x < NW) {
    float sw = 0.f, sb = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sw += red[0][k][threadIdx.x];
      sb += red[1][k][threadIdx.x];
    }
    tot[0][threadIdx.x] = sw;
    tot[1][threadIdx.x] = sb;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (a.splits > 1) {
    if (j < NW) {
      a.part[((int64_t)kk * a.splits + split) * NW + j] = tot[0][j];
      if (bias) a.bpart[(int64_t)split * NW + j] = tot[1][j];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t prev = atomicAdd(a.counters + kk, 1u);
      last = prev == (uint32_t)a.splits - 1;
      if (last) a.counters[kk] = 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (j < NW) {
      float sw = 0.f, sb = 0.f;
      for (int32_t q = 0; q < a.splits; ++q) {
        sw += __ldcg(a.part + ((int64_t)kk * a.splits + q) * NW + j);
        if (bias) sb += __ldcg(a.bpart + (int64_t)q * NW + j);
      }
      tot[0][j] = sw;
      tot[1][j] = sb;
    }
  }
  // tap-major [K][cout][cin]: weight j = (n, m) of tap kk
  if (j < nw && j < NW) a.dW[(int64_t)kk * nw + j] += tot[0][j];
  if (bias && j < a.cout && j < NW) a.db[j] += tot[1][j];
}

struct BwdMerge {
  int32_t op, chans, n, steps, u;
  Ring gy;  // adjoint of the merge's output (rows == 0: gy_ext)
  const float* gy_ext;
  int64_t gy_stride;
  int32_t nin;
  Ring in[3];      // FP32 forward views of the inputs (heads need the values)
  Ring gin[3];     // adjoint rings to add into (rows == 0: skip this input)
  int32_t A[3];
  int64_t delay;   // heads: noise key offset
  int32_t noise;
  Batch b;
  char* adj;
  int64_t adj_slot_bytes;
};

__device__ __forceinline__ float fwd_val(const Batch& b, int32_t s, const Ring& r, int64_t t, int32_t c) {
  return reinterpret_cast<const float*>(slot_base(b, s) + r.off)[ring_row(t, r.rows) * r.chans + r.choff + c];
}

__global__ void k_bwd_merge(BwdMerge a) {
  const int64_t total = (int64_t)a.b.count * a.n * a.chans;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(idx % a.chans);
    const int64_t q = idx / a.chans;
    const int32_t j = (int32_t)(q % a.n);
    const int32_t s = (int32_t)(q / a.n);
    const int64_t t = chunk_t0(a.b, s, a.u, a.steps) + j;
    const int32_t slot = a.b.slots[s];
    const float g = a.gy.rows ? adj_row(a.adj, a.adj_slot_bytes, slot, a.gy, t)[c]
                              : a.gy_ext[(int64_t)s * a.gy_stride + (int64_t)j * a.chans + c];
    if (a.op == CC_OP_ADD) {
      for (int k = 0; k < a.nin; ++k)
        if (a.gin[k].rows) adj_row(a.adj, a.adj_slot_bytes, slot, a.gin[k], t - a.A[k])[c] += g;
    } else {
      const float w = fwd_val(a.b, s, a.in[0], t - a.A[0], c);
      const float am = fwd_val(a.b, s, a.in[1], t - a.A[1], c);
      const float nz = fwd_val(a.b, s, a.in[2], t - a.A[2], c);
      const float th = tanhf(w), sa = 1.f / (1.f + expf(-am)), sn = 1.f / (1.f + expf(-nz));
      float u = 0.f;
      if (a.noise) u = noise_uniform(a.b.seeds[slot], t - a.delay, c, a.chans);
      const float gw = g * (1.f - th * th) * sa, ga = g * th * sa * (1.f - sa), gn = g * u * sn * (1.f - sn);
      const float gs[3] = {gw, ga, gn};
      for (int k = 0; k < 3; ++k)
        if (a.gin[k].rows) adj_row(a.adj, a.adj_slot_bytes, slot, a.gin[k], t - a.A[k])[c] += gs[k];
    }
  }
}

__global__ void k_adj_out(Batch b, char* adj, int64_t adj_slot_bytes, Ring r, int32_t n, int32_t steps, float* gx,
                          int64_t stride) {
  const int64_t total = (int64_t)b.count * n * r.chans;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i % r.chans);
    const int64_t q = i / r.chans;
    const int32_t j = (int32_t)(q % n);
    const int32_t s = (int32_t)(q / n);
    gx[(int64_t)s * stride + (int64_t)j * r.chans + c] =
        adj_row(adj, adj_slot_bytes, b.slots[s], r, chunk_t0(b, s, r.u, steps) + j)[c];
  }
}

int grid_of(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

// Splits of a reduction of `steps` steps over `tiles` output tiles, at least
// `min_steps` steps each, within the partial buffer; per_split is set to the
// steps of one split (a multiple of `align`).
int32_t pick_splits(int64_t tiles, int64_t steps, int64_t min_steps, int64_t align, int64_t* per_split) {
  int64_t sp = 1;
  if (tiles < kTargetBlocks) {
    sp = (kTargetBlocks + tiles - 1) / tiles;
    sp = std::min(sp, std::max<int64_t>(1, steps / min_steps));
    sp = std::min(sp, std::max<int64_t>(1, kPartTiles / tiles));
  }
  int64_t per = (steps + sp - 1) / sp;
  per = (per + align - 1) / align * align;
  *per_split = std::max<int64_t>(per, align);
  return (int32_t)std::max<int64_t>(1, (steps + *per_split - 1) / *per_split);
}

}  // namespace

// ===========================================================================
struct cc_grads {
  cc::Model* m = nullptr;
  char* adj = nullptr;          // adjoint arena: max_streams slots of adj_slot_bytes
  int64_t adj_slot_bytes = 0;
  std::vector<cc::Ring> adj_ring;  // per node: FP32 adjoint ring (rows 0: none)
  std::vector<float*> dW, db;
  std::vector<size_t> nW;
  std::vector<float*> Wt;  // per conv node: the weights the forward multiplied, [K][cout][cin]
  int32_t* d_slots = nullptr;
  int32_t* h_slots = nullptr;
  cudaEvent_t upload_done = nullptr;
  std::vector<int32_t> uploaded;  // the slot list d_slots holds
  // split-reduction scratch of the GEMM kernels (shared by their launches,
  // which run in order on the caller's stream)
  float* part = nullptr;
  float* bpart = nullptr;
  uint32_t* counters = nullptr;
  // measurement (cc_grads_timing): device time per kernel class and node
  struct TimingRec {
    int32_t cls, node;
    cudaEvent_t start, stop;
  };
  bool timing_on = false;
  std::vector<TimingRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  cudaError_t take_event(cudaEvent_t* e) {
    if (pool_used == pool.size()) {
      cudaEvent_t n = nullptr;
      const cudaError_t r = cudaEventCreate(&n);
      if (r != cudaSuccess) return r;
      pool.push_back(n);
    }
    *e = pool[pool_used++];
    return cudaSuccess;
  }
};

namespace {

// The weights a tensor-core layer multiplies: each packed GEMM row (an output
// channel of a convolution, a (phase, channel) row of a transposed one)
// scaled to max |w| = 1, rounded to the model's 16-bit type, scaled back.
void quantize_like_forward(const cc::Model& m, const cc_node_desc& d, std::vector<float>& w) {
  const bool bf16 = m.lp_dtype == cc::kDtBF16;
  auto round16 = [&](float x) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : __half2float(__float2half_rn(x));
  };
  if (d.op == CC_OP_CONV) {
    const size_t row = (size_t)d.c_in * d.kernel;
    for (int o = 0; o < d.c_out; ++o) {
      float mx = 0.f;
      for (size_t k = 0; k < row; ++k) mx = std::max(mx, std::fabs(w[o * row + k]));
      const float sc = mx > 0.f ? mx : 1.f;
      for (size_t k = 0; k < row; ++k) w[o * row + k] = round16(w[o * row + k] / sc) * sc;
    }
  } else {
    const int S = d.stride, T = d.kernel / S;
    for (int ph = 0; ph < S; ++ph)
      for (int o = 0; o < d.c_out; ++o) {
        float mx = 0.f;
        for (int c = 0; c < d.c_in; ++c)
          for (int j = 0; j < T; ++j) mx = std::max(mx, std::fabs(w[((size_t)c * d.c_out + o) * d.kernel + ph + j * S]));
        const float sc = mx > 0.f ? mx : 1.f;
        for (int c = 0; c < d.c_in; ++c)
          for (int j = 0; j < T; ++j) {
            float& x = w[((size_t)c * d.c_out + o) * d.kernel + ph + j * S];
            x = round16(x / sc) * sc;
          }
      }
  }
}

}  // namespace

extern "C" {

cc_status cc_grads_create(cc_model* model, const float* const* weights, cc_grads** out) {
  using cc::fail;
  if (!model || !out || !weights) return fail(CC_ERR_INVALID_ARG, "null argument");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (m->max_streams == 0) return fail(CC_ERR_STATE, "plan-only model");
  if (m->dtype != CC_F32 && m->fuse_units)
    return fail(CC_ERR_STATE,
                "a low-precision model is differentiable only with CC_FLAG_NO_UNIT_FUSION (a fused residual "
                "unit keeps its intermediate on chip, and the backward reads it)");
  for (size_t i = 0; i < m->nodes.size(); ++i) {
    const cc_node_desc& d = m->nodes[i].d;
    if ((d.op == CC_OP_CONV || d.op == CC_OP_CONVT) && !weights[i])
      return fail(CC_ERR_INVALID_ARG, "node %zu: missing weights", i);
  }
  auto* g = new cc_grads();
  g->m = m;
  const size_t n = m->nodes.size();
  g->dW.assign(n, nullptr);
  g->db.assign(n, nullptr);
  g->nW.assign(n, 0);
  g->Wt.assign(n, nullptr);
  g->adj_ring.assign(n, cc::Ring{});
  auto bad = [&](const char* what) {
    cudaGetLastError();
    for (size_t i = 0; i < n; ++i) {
      if (g->dW[i]) cudaFree(g->dW[i]);
      if (g->db[i]) cudaFree(g->db[i]);
      if (g->Wt[i]) cudaFree(g->Wt[i]);
    }
    if (g->adj) cudaFree(g->adj);
    if (g->part) cudaFree(g->part);
    if (g->bpart) cudaFree(g->bpart);
    if (g->counters) cudaFree(g->counters);
    if (g->d_slots) cudaFree(g->d_slots);
    if (g->h_slots) cudaFreeHost(g->h_slots);
    delete g;
    return fail(CC_ERR_NO_MEMORY, "gradient buffers: %s", what);
  };
  // adjoint arena: an FP32 ring per node that anything reads (its kept
  // history plus a call's frames), independent of the forward's views
  int64_t off = 0;
  for (size_t i = 0; i < n; ++i) {
    const cc::NodePlan& p = m->nodes[i];
    if (p.consumers.empty() && i + 1 != n) continue;
    cc::Ring r{};
    r.off = off;
    r.rows = p.keep + p.u * m->max_steps;
    r.chans = p.d.c_out;
    r.u = p.u;
    r.dtype = cc::kDtF32;
    g->adj_ring[i] = r;
    off += ((int64_t)r.rows * r.chans * 4 + 255) / 256 * 256;
  }
  g->adj_slot_bytes = std::max<int64_t>(off, 256);
  if (cudaMalloc(&g->part, (size_t)kPartTiles * kBT * kBT * 4) != cudaSuccess ||
      cudaMalloc(&g->bpart, (size_t)kPartTiles * kBT * 4) != cudaSuccess ||
      cudaMalloc(&g->counters, (size_t)2 * kPartTiles * 4) != cudaSuccess ||
      cudaMemset(g->counters, 0, (size_t)2 * kPartTiles * 4) != cudaSuccess)
    return bad("split-reduction scratch");
  if (cudaMalloc(&g->adj, (size_t)g->adj_slot_bytes * m->max_streams) != cudaSuccess) return bad("adjoint arena");
  if (cudaMemset(g->adj, 0, (size_t)g->adj_slot_bytes * m->max_streams) != cudaSuccess) return bad("adjoint arena");
  if (cudaMalloc(&g->d_slots, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
      cudaMallocHost(&g->h_slots, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->upload_done, cudaEventDisableTiming) != cudaSuccess)
    return bad("batch list");
  for (size_t i = 0; i < n; ++i) {
    const cc::NodePlan& p = m->nodes[i];
    const cc_node_desc& d = p.d;
    if (d.op != CC_OP_CONV && d.op != CC_OP_CONVT) continue;
    g->nW[i] = (size_t)d.c_in * d.c_out * d.kernel;
    std::vector<float> w(weights[i], weights[i] + g->nW[i]);
    if (p.engine == 1) quantize_like_forward(*m, d, w);
    // per tap [K][cout][cin]: conv W[n][m][k]; transposed conv W[m][n][k]
    std::vector<float> wt(g->nW[i]);
    for (int k = 0; k < d.kernel; ++k)
      for (int o = 0; o < d.c_out; ++o)
        for (int c = 0; c < d.c_in; ++c)
          wt[((size_t)k * d.c_out + o) * d.c_in + c] = d.op == CC_OP_CONV
                                                            ? w[((size_t)o * d.c_in + c) * d.kernel + k]
                                                            : w[((size_t)c * d.c_out + o) * d.kernel + k];
    if (cudaMalloc(&g->dW[i], g->nW[i] * 4) != cudaSuccess || cudaMalloc(&g->Wt[i], g->nW[i] * 4) != cudaSuccess)
      return bad("weight gradient");
    if (cudaMemcpy(g->Wt[i], wt.data(), g->nW[i] * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return bad("weight upload");
    if (d.has_bias && cudaMalloc(&g->db[i], (size_t)d.c_out * 4) != cudaSuccess) return bad("bias gradient");
  }
  *out = g;
  return cc_grads_zero(g);
}

cc_status cc_grads_destroy(cc_grads* g) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  cudaDeviceSynchronize();
  for (size_t i = 0; i < g->dW.size(); ++i) {
    if (g->dW[i]) cudaFree(g->dW[i]);
    if (g->db[i]) cudaFree(g->db[i]);
    if (g->Wt[i]) cudaFree(g->Wt[i]);
  }
  cudaFree(g->adj);
  cudaFree(g->part);
  cudaFree(g->bpart);
  cudaFree(g->counters);
  cudaFree(g->d_slots);
  cudaFreeHost(g->h_slots);
  cudaEventDestroy(g->upload_done);
  for (cudaEvent_t e : g->pool) cudaEventDestroy(e);
  delete g;
  return CC_OK;
}

cc_status cc_grads_timing(cc_grads* g, int32_t enable) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  if (cudaDeviceSynchronize() != cudaSuccess) return cc::fail(CC_ERR_CUDA, "synchronize failed");
  g->timing_on = enable != 0;
  g->recs.clear();
  g->pool_used = 0;
  return CC_OK;
}

cc_status cc_grads_timing_read(cc_grads* g, double* ms, int64_t* launches, int32_t n_classes) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  if (n_classes != CC_BWD_CLASSES) return cc::fail(CC_ERR_INVALID_ARG, "n_classes must be %d", CC_BWD_CLASSES);
  for (int i = 0; i < n_classes; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  for (auto& r : g->recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess)
      return cc::fail(CC_ERR_CUDA, "timing read failed");
    if (ms) ms[r.cls] += t;
    if (launches) launches[r.cls] += 1;
  }
  return CC_OK;
}

cc_status cc_grads_timing_read_nodes(cc_grads* g, int32_t n_nodes, double* ms, int64_t* launches) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  if (n_nodes != (int32_t)g->m->nodes.size()) return cc::fail(CC_ERR_INVALID_ARG, "n_nodes mismatch");
  const size_t total = (size_t)n_nodes * CC_BWD_CLASSES;
  for (size_t i = 0; i < total; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  for (auto& r : g->recs) {
    if (r.node < 0) continue;
    float t = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess)
      return cc::fail(CC_ERR_CUDA, "timing read failed");
    if (ms) ms[(size_t)r.node * CC_BWD_CLASSES + r.cls] += t;
    if (launches) launches[(size_t)r.node * CC_BWD_CLASSES + r.cls] += 1;
  }
  return CC_OK;
}

cc_status cc_grads_zero(cc_grads* g) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  for (size_t i = 0; i < g->dW.size(); ++i) {
    if (g->dW[i] && cudaMemset(g->dW[i], 0, g->nW[i] * 4) != cudaSuccess)
      return cc::fail(CC_ERR_CUDA, "memset failed");
    if (g->db[i] && cudaMemset(g->db[i], 0, (size_t)g->m->nodes[i].d.c_out * 4) != cudaSuccess)
      return cc::fail(CC_ERR_CUDA, "memset failed");
  }
  return CC_OK;
}

cc_status cc_grads_read(cc_grads* g, int32_t node, float* dw, float* db) {
  if (!g) return cc::fail(CC_ERR_INVALID_ARG, "null gradients");
  if (node < 0 || node >= (int32_t)g->dW.size() || !g->dW[node])
    return cc::fail(CC_ERR_INVALID_ARG, "node %d has no weights", node);
  if (cudaDeviceSynchronize() != cudaSuccess) return cc::fail(CC_ERR_CUDA, "synchronize failed");
  if (dw) {
    // accumulated tap-major [K][cout][cin]; the trained layout is [cout][cin][K]
    // (conv) or [cin][cout][K] (transposed conv)
    const cc_node_desc& d = g->m->nodes[node].d;
    std::vector<float> t(g->nW[node]);
    if (cudaMemcpy(t.data(), g->dW[node], g->nW[node] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return cc::fail(CC_ERR_CUDA, "copy failed");
    for (int k = 0; k < d.kernel; ++k)
      for (int o = 0; o < d.c_out; ++o)
        for (int c = 0; c < d.c_in; ++c)
          dw[d.op == CC_OP_CONV ? ((size_t)o * d.c_in + c) * d.kernel + k : ((size_t)c * d.c_out + o) * d.kernel + k] =
              t[((size_t)k * d.c_out + o) * d.c_in + c];
  }
  if (db && g->db[node] &&
      cudaMemcpy(db, g->db[node], (size_t)g->m->nodes[node].d.c_out * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cc::fail(CC_ERR_CUDA, "copy failed");
  return CC_OK;
}

cc_status cc_backward_begin(cc_grads* g, cc_stream* const* streams, int32_t count, void* cuda_stream) {
  if (!g || !streams || count < 0) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  for (int32_t i = 0; i < count; ++i) {
    if (!streams[i] || cc::stream_model(streams[i]) != g->m) return cc::fail(CC_ERR_INVALID_ARG, "stream %d", i);
    if (cc::stream_manipulated(streams[i]))
      return cc::fail(CC_ERR_STATE, "stream %d has an input manipulation; the backward does not differentiate it", i);
    const cudaError_t e = cudaMemsetAsync(g->adj + (size_t)cc::stream_slot(streams[i]) * g->adj_slot_bytes, 0,
                                          (size_t)g->adj_slot_bytes, st);
    if (e != cudaSuccess) return cc::fail(CC_ERR_CUDA, "adjoint reset: %s", cudaGetErrorString(e));
  }
  return CC_OK;
}

cc_status cc_backward_chunk(cc_grads* g, cc_stream* const* streams, int32_t count, const float* x,
                            int64_t x_stride, int64_t n_in, const float* grad_y, int64_t gy_stride,
                            int64_t n_out, float* grad_x, int64_t gx_stride, void* cuda_stream) {
  using cc::fail;
  if (!g || !streams || count <= 0 || !x || !grad_y) return fail(CC_ERR_INVALID_ARG, "null argument");
  cc::Model* m = g->m;
  if (count > m->max_streams) return fail(CC_ERR_INVALID_ARG, "batch larger than max_streams");
  if (n_in <= 0 || n_in % m->in_per_step) return fail(CC_ERR_BAD_LENGTH, "n_in must be a positive multiple of the model step");
  const int64_t steps64 = n_in / m->in_per_step;
  if (steps64 > m->max_steps) return fail(CC_ERR_BAD_LENGTH, "a backward chunk is at most max_steps_per_call steps");
  const int32_t steps = (int32_t)steps64;
  if (n_out != steps64 * m->nodes.back().u) return fail(CC_ERR_BAD_LENGTH, "n_out does not match n_in");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
#define BW_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(CC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
  // batch list: uploaded again only when it changed (the pinned staging may
  // still feed the previous upload)
  std::vector<int32_t> slots(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!streams[i] || cc::stream_model(streams[i]) != m) return fail(CC_ERR_INVALID_ARG, "stream %d", i);
    if (cc::stream_manipulated(streams[i]))
      return fail(CC_ERR_STATE, "stream %d has an input manipulation; the backward does not differentiate it", i);
    slots[i] = cc::stream_slot(streams[i]);
  }
  if (slots != g->uploaded) {
    BW_CUDA(cudaEventSynchronize(g->upload_done));
    std::memcpy(g->h_slots, slots.data(), sizeof(int32_t) * count);
    BW_CUDA(cudaMemcpyAsync(g->d_slots, g->h_slots, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
    BW_CUDA(cudaEventRecord(g->upload_done, st));
    g->uploaded = slots;
  }
  const cc::Batch b = m->batch_for(g->d_slots, count);
  auto t_begin = [&](int32_t cls, int32_t node) -> cudaError_t {
    if (!g->timing_on) return cudaSuccess;
    cc_grads::TimingRec r{cls, node, nullptr, nullptr};
    cudaError_t e = g->take_event(&r.start);
    if (e == cudaSuccess) e = g->take_event(&r.stop);
    if (e == cudaSuccess) e = cudaEventRecord(r.start, st);
    if (e == cudaSuccess) g->recs.push_back(r);
    return e;
  };
  auto t_end = [&]() -> cudaError_t {
    return g->timing_on ? cudaEventRecord(g->recs.back().stop, st) : cudaSuccess;
  };
  // 1. recompute this chunk's forward from the restored state; its output is
  //    not needed (grad_x doubles as scratch only if the shapes agree, so use
  //    the model's staging buffers)
  cc::Model::Staging* sg = nullptr;
  cc_status s = m->ensure_staging(count, st, &sg);
  if (s) return s;
  BW_CUDA(t_begin(CC_BWD_RECOMPUTE, -1));
  s = m->run_chain(b, x, x_stride, sg->out, (int64_t)steps * m->nodes.back().u * m->nodes.back().d.c_out,
                   steps, st);
  if (s) return s;
  BW_CUDA(t_end());
  // 2. clear the adjoint rows no later chunk could have written (the model
  //    input's only when its adjoint is wanted)
  const int n = (int)m->nodes.size();
  {
    ClearList L{};
    auto flush = [&]() -> cudaError_t {
      if (!L.count) return cudaSuccess;
      cudaError_t e = t_begin(CC_BWD_CLEAR, -1);
      if (e != cudaSuccess) return e;
      k_adj_clear<<<grid_of(L.start[L.count]), 256, 0, st>>>(b, g->adj, g->adj_slot_bytes, L, steps);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = t_end();
      L.count = 0;
      return e;
    };
    for (int i = 0; i < n; ++i) {
      const cc::NodePlan& p = m->nodes[i];
      const cc::Ring& r = g->adj_ring[i];
      if (!r.rows || (i == 0 && !grad_x)) continue;
      const int32_t k = L.count;
      L.r[k] = r;
      L.keep[k] = p.keep;
      L.n[k] = p.u * steps;
      L.start[k + 1] = L.start[k] + (int64_t)count * L.n[k] * r.chans;
      if (++L.count == kClearMax) BW_CUDA(flush());
    }
    BW_CUDA(flush());
  }
  // 3. nodes in reverse order
  auto gy_ring = [&](int wi) -> cc::Ring { return wi == n - 1 ? cc::Ring{} : g->adj_ring[wi]; };
  const int32_t lp_bf16 = m->lp_dtype == cc::kDtBF16;
  for (int i = n - 1; i >= 1; --i) {
    const cc::NodePlan& p = m->nodes[i];
    const cc_node_desc& d = p.d;
    if (d.op == CC_OP_CONV || d.op == CC_OP_CONVT) {
      const int wi = p.fused_add >= 0 ? p.fused_add : i;
      if (wi != n - 1 && !g->adj_ring[wi].rows) continue;  // dead branch: zero adjoint
      const cc::NodePlan& src = m->nodes[d.inputs[0]];
      BwdConv a{};
      a.Wt = g->Wt[i];
      a.op = d.op;
      a.cin = d.c_in;
      a.cout = d.c_out;
      a.K = d.kernel;
      a.S = d.stride;
      a.dil = d.op == CC_OP_CONV ? d.dilation : 1;
      a.hist = p.hist_need;
      a.n_in = src.u * steps;
      a.n_out = m->nodes[wi].u * steps;
      // the values the forward multiplied: the low-precision view a tensor-core
      // layer read (activation pre-applied), else the FP32 view
      if (p.engine == 1) {
        a.x.r = src.view[1 + d.act_in];
        a.x.kind = 1 + d.act_in;
      } else {
        a.x.r = src.view[0];
        a.x.kind = 0;
      }
      a.x.act = d.act_in;
      a.x.lp_bf16 = lp_bf16;
      a.u_in = src.u;
      a.u_out = m->nodes[wi].u;
      a.gy = gy_ring(wi);
      a.gy_ext = grad_y;
      a.gy_stride = gy_stride;
      a.gx = g->adj_ring[d.inputs[0]];
      a.dW = g->dW[i];
      a.db = g->db[i];
      a.steps = steps;
      a.b = b;
      a.adj = g->adj;
      a.adj_slot_bytes = g->adj_slot_bytes;
      a.part = g->part;
      a.bpart = g->bpart;
      a.counters = g->counters;
      const int64_t tm = (a.cin + kBT - 1) / kBT, tn = (a.cout + kBT - 1) / kBT;
      const bool narrow = a.cin < 16 || a.cout < 16;
      // dL/dx (not needed for the model input when the caller wants no grad_x)
      if (grad_x || d.inputs[0] != 0) {
        BW_CUDA(t_begin(CC_BWD_DATA, i));
        if (narrow) {
          k_bwd_data_narrow<<<grid_of((int64_t)count * (a.hist + a.n_in) * a.cin), 256, 0, st>>>(a);
        } else {
          // (stream, frame) row tiles x input-channel tiles, the (tap,
          // 32-channel chunk) reduction split
          const int64_t span = a.hist + a.n_in;
          int64_t rt = ((int64_t)count * span + kBT - 1) / kBT, taps = a.K;
          a.res = d.op == CC_OP_CONV && a.S > 1 && a.dil == 1;
          if (a.res) {
            rt = 0;
            for (int32_t r = 0; r < a.S; ++r) rt += ((int64_t)count * ((span - r + a.S - 1) / a.S) + kBT - 1) / kBT;
            taps = (a.K + a.S - 1) / a.S;
          }
          a.splits = pick_splits(rt * tm, taps * ((a.cout + kBC - 1) / kBC), 4, 1, &a.per_split);
          k_bwd_data<<<dim3((unsigned)rt, (unsigned)tm, (unsigned)a.splits), 256, 0, st>>>(a);
        }
        BW_CUDA(cudaGetLastError());
        BW_CUDA(t_end());
      }
      // dL/dW (and dL/db)
      BW_CUDA(t_begin(CC_BWD_WEIGHT, i));
      if (narrow && a.cout * a.cin <= 64) {
        // blocks over (tap, split of the columns)
        const int64_t cols = (int64_t)count * (d.op == CC_OP_CONVT ? a.n_in : a.n_out);
        a.splits = pick_splits(a.K, cols, 256, 1, &a.per_split);
        const dim3 grid((unsigned)a.K, (unsigned)a.splits);
        if (a.cout * a.cin <= 16)
          k_bwd_weight_tap<16><<<grid, 256, 0, st>>>(a);
        else
          k_bwd_weight_tap<64><<<grid, 256, 0, st>>>(a);
      } else if (narrow) {
        k_bwd_weight_narrow<<<(unsigned)((int64_t)a.cout * a.cin * a.K), 256, 0, st>>>(a);
      } else {
        // output-channel x input-channel x tap tiles, the (stream, frame)
        // columns split
        const int64_t cols = (int64_t)count * (d.op == CC_OP_CONVT ? a.n_in : a.n_out);
        a.splits = pick_splits(tn * tm * a.K, cols, 2 * kBC, kBC, &a.per_split);
        // bias partials: (output-channel tile, phase, split) within the buffer
        const int64_t nph = d.op == CC_OP_CONVT ? a.S : 1;
        if (a.db && tn * nph * a.splits > kPartTiles) {
          if (tn * nph > kPartTiles)
            return fail(CC_ERR_INVALID_ARG, "node %d: too many output channels x phases for the bias reduction", i);
          a.splits = (int32_t)(kPartTiles / (tn * nph));
          a.per_split = ((cols + a.splits - 1) / a.splits + kBC - 1) / kBC * kBC;
          a.splits = (int32_t)((cols + a.per_split - 1) / a.per_split);
        }
        k_bwd_weight<<<dim3((unsigned)tn, (unsigned)tm, (unsigned)(a.K * a.splits)), 256, 0, st>>>(a);
      }
      BW_CUDA(cudaGetLastError());
      BW_CUDA(t_end());
    } else if (d.op == CC_OP_ADD || d.op == CC_OP_HEADS) {
      if (i != n - 1 && !g->adj_ring[i].rows) continue;  // dead branch
      BwdMerge a{};
      a.op = d.op;
      a.chans = d.c_out;
      a.n = p.u * steps;
      a.steps = steps;
      a.u = p.u;
      a.gy = gy_ring(i);
      a.gy_ext = grad_y;
      a.gy_stride = gy_stride;
      a.nin = d.n_inputs;
      for (int k = 0; k < d.n_inputs; ++k) {
        const int src = d.inputs[k];
        a.in[k] = m->nodes[src].view[0];
        // a fused add's conv reads the add's adjoint directly
        const bool into_conv = p.fused && m->nodes[src].fused_add == i;
        a.gin[k] = into_conv ? cc::Ring{} : g->adj_ring[src];
        a.A[k] = p.A[k];
      }
      a.delay = p.D;
      a.noise = m->noise;
      a.b = b;
      a.adj = g->adj;
      a.adj_slot_bytes = g->adj_slot_bytes;
      BW_CUDA(t_begin(CC_BWD_MERGE, i));
      k_bwd_merge<<<grid_of((int64_t)count * a.n * a.chans), 256, 0, st>>>(a);
      BW_CUDA(cudaGetLastError());
      BW_CUDA(t_end());
    }
  }
  // 4. the input adjoint of this chunk's frames
  if (grad_x) {
    const cc::NodePlan& p0 = m->nodes[0];
    BW_CUDA(t_begin(CC_BWD_INPUT, 0));
    k_adj_out<<<grid_of((int64_t)count * p0.u * steps * p0.d.c_out), 256, 0, st>>>(
        b, g->adj, g->adj_slot_bytes, g->adj_ring[0], p0.u * steps, steps, grad_x, gx_stride);
    BW_CUDA(cudaGetLastError());
    BW_CUDA(t_end());
  }
#undef BW_CUDA
  return CC_OK;
}

cc_status cc_model_snapshot_bytes(const cc_model* model, size_t* bytes) {
  if (!model || !bytes) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  *bytes = reinterpret_cast<const cc::Model*>(model)->snapshot_bytes;
  return CC_OK;
}

}  // extern "C"

namespace {

// Copies the cached state of `count` streams between their arena slots and a
// compact buffer (stream i at buf + i * snap_bytes: step counter, noise seed,
// then each region's kept rows, oldest first), four bytes per thread.
// Restoring also rewrites the mirrored copy of a low-precision view's tail.
__global__ void k_state_copy(cc::Batch b, const cc::Model::StateRegion* regs, int32_t n_regs, char* buf,
                             int64_t snap_bytes, int32_t to_slots) {
  const int64_t words = snap_bytes / 4;
  const int64_t per = n_regs ? words : 4;  // no regions: the counter and seed words only
  const int64_t total = (int64_t)b.count * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(i / per);
    int64_t w = i - (int64_t)s * per;
    const int32_t slot = b.slots[s];
    uint32_t* bw = reinterpret_cast<uint32_t*>(buf + (int64_t)s * snap_bytes) + w;
    if (w < 4) {  // counter, seed
      uint32_t* src = w < 2 ? reinterpret_cast<uint32_t*>(const_cast<int64_t*>(b.counters) + slot) + w
                            : reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(b.seeds) + slot) + (w - 2);
      if (to_slots)
        *src = *bw;
      else
        *bw = *src;
      continue;
    }
    w -= 4;
    int32_t k = 0;
    for (; k < n_regs; ++k) {
      const int64_t rw = (int64_t)regs[k].keep * regs[k].row_bytes / 4;
      if (w < rw) break;
      w -= rw;
    }
    if (k >= n_regs) continue;
    const cc::Model::StateRegion& g = regs[k];
    const int32_t per_row = g.row_bytes / 4;
    const int32_t q = (int32_t)(w / per_row), c = (int32_t)(w - (int64_t)q * per_row);
    // the step counter in the buffer is the state's: at restore it is the one
    // being written (read it from the buffer), at snapshot the slot's
    const int64_t steps = *reinterpret_cast<const int64_t*>(buf + (int64_t)s * snap_bytes);
    const int64_t t = steps * g.u - g.keep + q;
    const int64_t row = ring_row(t, g.rows);
    uint32_t* slot_word = reinterpret_cast<uint32_t*>(b.arena + (int64_t)slot * b.slot_bytes + g.off + row * g.row_bytes) + c;
    if (to_slots) {
      *slot_word = *bw;
      if (g.pre && row >= g.rows - g.pre)
        *reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(slot_word) - (int64_t)g.rows * g.row_bytes) = *bw;
    } else {
      *bw = *slot_word;
    }
  }
}

cc_status state_copy(cc::Model* m, cc_stream* const* streams, int32_t count, void* buf, size_t bytes, int32_t to_slots,
                     cudaStream_t st) {
  using cc::fail;
  if (!streams || !buf || count <= 0) return fail(CC_ERR_INVALID_ARG, "null argument or empty batch");
  if (count > m->max_streams) return fail(CC_ERR_INVALID_ARG, "batch larger than max_streams");
  if (bytes != (size_t)count * m->snapshot_bytes)
    return fail(CC_ERR_INVALID_ARG, "snapshot buffer must hold %d x %zu bytes", count, m->snapshot_bytes);
  if (reinterpret_cast<uintptr_t>(buf) % 8) return fail(CC_ERR_INVALID_ARG, "snapshot buffer must be 8-byte aligned");
  std::vector<int32_t> slots(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!streams[i] || cc::stream_model(streams[i]) != m) return fail(CC_ERR_INVALID_ARG, "stream %d not of this model", i);
    slots[i] = cc::stream_slot(streams[i]);
  }
  const int32_t* d_list = nullptr;
  cc_status r = cc::upload_slot_list(m, slots, st, &d_list);
  if (r) return r;
  const cc::Batch b = m->batch_for(d_list, count);
  if (!to_slots) {
    // the counters first (every state row's time depends on them), then the rows
    k_state_copy<<<(count * 4 + 255) / 256, 256, 0, st>>>(b, m->d_state_regions, 0, static_cast<char*>(buf),
                                                        (int64_t)m->snapshot_bytes, 0);
    if (cudaGetLastError() != cudaSuccess) return fail(CC_ERR_CUDA, "snapshot launch failed");
  }
  k_state_copy<<<grid_of((int64_t)count * m->snapshot_bytes / 4), 256, 0, st>>>(
      b, m->d_state_regions, (int32_t)m->state_regions.size(), static_cast<char*>(buf), (int64_t)m->snapshot_bytes,
      to_slots);
  if (cudaGetLastError() != cudaSuccess) return fail(CC_ERR_CUDA, "state copy launch failed");
  return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_snapshot_batch(cc_model* model, cc_stream* const* streams, int32_t count, void* dev_buf, size_t bytes,
                            void* cuda_stream) {
  if (!model) return cc::fail(CC_ERR_INVALID_ARG, "null model");
  return state_copy(reinterpret_cast<cc::Model*>(model), streams, count, dev_buf, bytes, 0,
                    reinterpret_cast<cudaStream_t>(cuda_stream));
}

cc_status cc_restore_batch(cc_model* model, cc_stream* const* streams, int32_t count, const void* dev_buf, size_t bytes,
                           void* cuda_stream) {
  if (!model) return cc::fail(CC_ERR_INVALID_ARG, "null model");
  return state_copy(reinterpret_cast<cc::Model*>(model), streams, count, const_cast<void*>(dev_buf), bytes, 1,
                    reinterpret_cast<cudaStream_t>(cuda_stream));
}

cc_status cc_stream_snapshot(cc_stream* s, void* dev, size_t bytes, void* cuda_stream) {
  if (!s) return cc::fail(CC_ERR_INVALID_ARG, "null stream");
  return state_copy(cc::stream_model(s), &s, 1, dev, bytes, 0, reinterpret_cast<cudaStream_t>(cuda_stream));
}

cc_status cc_stream_restore(cc_stream* s, const void* dev, size_t bytes, void* cuda_stream) {
  if (!s) return cc::fail(CC_ERR_INVALID_ARG, "null stream");
  return state_copy(cc::stream_model(s), &s, 1, const_cast<void*>(dev), bytes, 1,
                    reinterpret_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"
