// FP32 kernels of the streamed model: cached convolutions (Eq. 1 over a ring
// window, section 2.2), polyphase transposed convolutions, the aligned merges
// (Eq. 3) and the RAVE-like heads.  The FP32 path is FFMA only: no TF32.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {
namespace {

// Epilogue of a conv / convT GEMM element: bias, fused residual (Eq. 3 aligned
// skip), store into every output view.
__device__ __forceinline__ void store_conv(const ConvArgs& a, int32_t m, int32_t n, float v) {
  const int32_t s = n / a.ncols;
  const int32_t j = n - s * a.ncols;
  int32_t ch, lt;
  if (a.phases == 1) {
    ch = m;
    lt = j;
  } else {
    const int32_t ph = m / a.cout;
    ch = m - ph * a.cout;
    lt = j * a.phases + ph;
  }
  if (a.bias) v += a.bias[ch];
  const int64_t t = steps_of(a.batch, s) * a.out_u + lt;
  if (a.has_skip) {
    const float* sk = ring_ptr<const float>(a.batch, s, a.skip);
    v += sk[ring_row(t - a.skip_A, a.skip.rows) * a.skip.chans + a.skip.choff + ch];
  }
  store_views(a.batch, s, a.out, t, lt, ch, a.cout, v);
}

// Epilogue of TM rows of one GEMM column (rows come in groups of four
// consecutive output rows): the column's ring rows are computed once (one
// modulo per view), every bias / residual load is issued before the first
// store, then the values go to every output view -- as float4 / 4-element
// low-precision stores when the channel count allows it.
// Ring rows of a column's first output time in each view (and of its
// residual): known from the stream's step counter alone, so the narrow kernel
// computes them before its dependency wait.
struct ColRows {
  int32_t rf, r0, r1, rs;
};

__device__ __forceinline__ ColRows col_rows(const ConvArgs& a, int64_t step, int32_t j) {
  const int64_t tb = step * a.out_u + (int64_t)j * a.phases;
  ColRows r;
  r.rf = a.out.f32.rows ? (int32_t)ring_row(tb, a.out.f32.rows) : 0;
  r.r0 = a.out.lp[0].rows ? (int32_t)ring_row(tb, a.out.lp[0].rows) : 0;
  r.r1 = a.out.lp[1].rows ? (int32_t)ring_row(tb, a.out.lp[1].rows) : 0;
  r.rs = a.has_skip ? (int32_t)ring_row(tb - a.skip_A, a.skip.rows) : 0;
  return r;
}

template <int TM>
__device__ __forceinline__ void store_column_rows(const ConvArgs& a, int32_t s, int32_t j, char* base,
                                                  const ColRows& cr, const int32_t (&m)[TM], float (&v)[TM],
                                                  bool vec) {
  const int32_t rf = cr.rf, r0 = cr.r0, r1 = cr.r1, rs = cr.rs;
  int32_t ph[TM], ch[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    ph[i] = a.phases == 1 ? 0 : m[i] / a.cout;
    ch[i] = m[i] - ph[i] * a.cout;
  }
  float add[TM];
  if (vec) {
#pragma unroll
    for (int g = 0; g < TM; g += 4) {
      float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m[g] < a.M) {
        if (a.bias) b4 = __ldg(reinterpret_cast<const float4*>(a.bias + ch[g]));
        if (a.has_skip) {
          const float4 s4 = __ldg(reinterpret_cast<const float4*>(
              reinterpret_cast<const float*>(base + a.skip.off) +
              (int64_t)wrap_row(rs + ph[g], a.skip.rows) * a.skip.chans + a.skip.choff + ch[g]));
          b4.x += s4.x; b4.y += s4.y; b4.z += s4.z; b4.w += s4.w;
        }
      }
      add[g] = b4.x; add[g + 1] = b4.y; add[g + 2] = b4.z; add[g + 3] = b4.w;
    }
#pragma unroll
    for (int g = 0; g < TM; g += 4) {
      if (m[g] >= a.M) continue;
      float x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = v[g + k] + add[g + k];
      if (a.out.f32.rows)
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(base + a.out.f32.off) +
                                   (int64_t)wrap_row(rf + ph[g], a.out.f32.rows) * a.out.f32.chans + ch[g]) =
            make_float4(x[0], x[1], x[2], x[3]);
      if (a.out.ext) {
        float* e = a.out.ext + (int64_t)s * a.out.ext_stride + ((int64_t)j * a.phases + ph[g]) * a.cout + ch[g];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = x[k];
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const Ring& lr = a.out.lp[q];
        if (!lr.rows) continue;
        const int32_t row = wrap_row((q ? r1 : r0) + ph[g], lr.rows);
#pragma unroll
        for (int k = 0; k < 4; ++k) store_lp(base, lr, row, ch[g] + k, q ? leaky(x[k]) : x[k]);
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    add[i] = 0.f;
    if (m[i] < a.M) {
      if (a.bias) add[i] = __ldg(a.bias + ch[i]);
      if (a.has_skip)
        add[i] += __ldg(reinterpret_cast<const float*>(base + a.skip.off) +
                        (int64_t)wrap_row(rs + ph[i], a.skip.rows) * a.skip.chans + a.skip.choff + ch[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    if (m[i] >= a.M) continue;
    const float x = v[i] + add[i];
    if (a.out.ext) a.out.ext[(int64_t)s * a.out.ext_stride + ((int64_t)j * a.phases + ph[i]) * a.cout + ch[i]] = x;
    if (a.out.f32.rows)
      reinterpret_cast<float*>(base + a.out.f32.off)[(int64_t)wrap_row(rf + ph[i], a.out.f32.rows) *
                                                         a.out.f32.chans + ch[i]] = x;
    if (a.out.lp[0].rows) store_lp(base, a.out.lp[0], wrap_row(r0 + ph[i], a.out.lp[0].rows), ch[i], x);
    if (a.out.lp[1].rows) store_lp(base, a.out.lp[1], wrap_row(r1 + ph[i], a.out.lp[1].rows), ch[i], leaky(x));
  }
}

template <int TM>
__device__ __forceinline__ void store_column(const ConvArgs& a, int32_t n, const int32_t (&m)[TM],
                                             float (&v)[TM], bool vec) {
  const int32_t s = n / a.ncols;
  const int32_t j = n - s * a.ncols;
  store_column_rows<TM>(a, s, j, slot_base(a.batch, s), col_rows(a, steps_of(a.batch, s), j), m, v, vec);
}

// ---------------------------------------------------------------------------
// Skinny GEMM (few columns per launch: single-stream steps).  One warp per
// output row m, eight columns per block column; the reduction over (tap,
// channel) is split across lanes and finished with warp shuffles.
// ---------------------------------------------------------------------------
constexpr int kGemvCols = 8;
constexpr int kGemvWarps = 8;

template <bool kVec>
__global__ void __launch_bounds__(kGemvWarps * 32) k_conv_gemv_f32(const ConvArgs a) {
  pdl_wait();
  pdl_release();
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t m = blockIdx.y * kGemvWarps + warp;
  const int32_t n0 = blockIdx.x * kGemvCols;
  const int32_t N = a.batch.count * a.ncols;
  if (m >= a.M) return;

  const float* col[kGemvCols];
  int32_t r0[kGemvCols];
  bool ok[kGemvCols];
#pragma unroll
  for (int c = 0; c < kGemvCols; ++c) {
    const int32_t n = n0 + c;
    ok[c] = n < N;
    col[c] = nullptr;
    r0[c] = 0;
    if (ok[c]) {
      const int32_t s = n / a.ncols, j = n - s * a.ncols;
      const int64_t t = steps_of(a.batch, s) * a.in.u + (int64_t)j * a.stride - a.hist;
      r0[c] = (int32_t)ring_row(t, a.in.rows);
      col[c] = ring_ptr<const float>(a.batch, s, a.in) + a.in.choff;
    }
  }
  float acc[kGemvCols];
#pragma unroll
  for (int c = 0; c < kGemvCols; ++c) acc[c] = 0.f;
  const float* Arow = a.A + (int64_t)m * a.Kt;

  if (kVec) {
    for (int32_t tap = 0; tap < a.taps; ++tap) {
      int32_t rowoff[kGemvCols];
#pragma unroll
      for (int c = 0; c < kGemvCols; ++c)
        rowoff[c] = wrap_row(r0[c] + tap * a.dil, a.in.rows) * a.in.chans;
      const float* At = Arow + tap * a.cin;
      for (int32_t ch = lane * 4; ch < a.cin; ch += 128) {
        const float4 w = *reinterpret_cast<const float4*>(At + ch);
#pragma unroll
        for (int c = 0; c < kGemvCols; ++c) {
          if (ok[c]) {
            const float4 x = *reinterpret_cast<const float4*>(col[c] + rowoff[c] + ch);
            acc[c] = fmaf(w.x, activate(x.x, a.act), acc[c]);
            acc[c] = fmaf(w.y, activate(x.y, a.act), acc[c]);
            acc[c] = fmaf(w.z, activate(x.z, a.act), acc[c]);
            acc[c] = fmaf(w.w, activate(x.w, a.act), acc[c]);
          }
        }
      }
    }
  } else {
    for (int32_t k = lane; k < a.Kt; k += 32) {
      const int32_t tap = k / a.cin, ch = k - tap * a.cin;
      const float w = Arow[k];
#pragma unroll
      for (int c = 0; c < kGemvCols; ++c) {
        if (ok[c]) {
          const int32_t row = wrap_row(r0[c] + tap * a.dil, a.in.rows);
          acc[c] = fmaf(w, activate(col[c][row * a.in.chans + ch], a.act), acc[c]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kGemvCols; ++c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  }
  float v = acc[0];
#pragma unroll
  for (int c = 1; c < kGemvCols; ++c)
    if (lane == c) v = acc[c];
  if (lane < kGemvCols && n0 + lane < N) store_conv(a, m, n0 + lane, v);
}

// ---------------------------------------------------------------------------
// Tiled GEMM (many columns: batched streams).  BM x BN tile, BK-deep K slices
// staged through shared memory (double-buffered via registers), 256 threads
// as a 16 x 16 grid, each computing (BM/16) x (BN/16) outputs.  With 8x8
// outputs a thread takes two groups of four rows (and columns) half a tile
// apart, so its float4 shared-memory reads stay conflict-free.
// Requires cin % BK == 0 so that a K slice lies inside one tap.
// ---------------------------------------------------------------------------
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_conv_tile_f32(const ConvArgs a) {
  constexpr int TM = BM / 16, TN = BN / 16;  // 4 or 8
  constexpr int GM = TM / 4, GN = TN / 4;    // groups of four
  constexpr int A4 = BM * BK / 4 / 256, B4 = BN * BK / 4 / 256;  // float4 per thread
  static_assert(A4 >= 1 && B4 >= 1, "tile too small for 256 threads");
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  pdl_wait();
  pdl_release();
  const int32_t tid = threadIdx.x;
  const int32_t tx = tid & 15, ty = tid >> 4;
  const int32_t m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int32_t N = a.batch.count * a.ncols;

  // loader coordinates
  int32_t lrowA[A4], lkA[A4], lrowB[B4], lkB[B4];
  const float* Arow[A4];
  bool a_ok[A4], b_ok[B4];
  const float* bcol[B4];
  int32_t br0[B4];
#pragma unroll
  for (int q = 0; q < A4; ++q) {
    const int f = tid + q * 256;
    lrowA[q] = f / (BK / 4);
    lkA[q] = (f % (BK / 4)) * 4;
    a_ok[q] = (m0 + lrowA[q]) < a.M;
    Arow[q] = a.A + (int64_t)(a_ok[q] ? m0 + lrowA[q] : 0) * a.Kt;
  }
#pragma unroll
  for (int q = 0; q < B4; ++q) {
    const int f = tid + q * 256;
    lrowB[q] = f / (BK / 4);
    lkB[q] = (f % (BK / 4)) * 4;
    const int32_t n = n0 + lrowB[q];
    b_ok[q] = n < N;
    bcol[q] = nullptr;
    br0[q] = 0;
    if (b_ok[q]) {
      const int32_t s = n / a.ncols, j = n - s * a.ncols;
      const int64_t t = steps_of(a.batch, s) * a.in.u + (int64_t)j * a.stride - a.hist;
      br0[q] = (int32_t)ring_row(t, a.in.rows);
      bcol[q] = ring_ptr<const float>(a.batch, s, a.in) + a.in.choff;
    }
  }
  float4 ra[A4], rb[B4];
  auto load = [&](int32_t kt) {
    const int32_t tap = kt / a.cin, chb = kt - tap * a.cin;
#pragma unroll
    for (int q = 0; q < A4; ++q)
      ra[q] = a_ok[q] ? *reinterpret_cast<const float4*>(Arow[q] + kt + lkA[q])
                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      if (b_ok[q]) {
        const int32_t row = wrap_row(br0[q] + tap * a.dil, a.in.rows);
        const float4 x =
            *reinterpret_cast<const float4*>(bcol[q] + (int64_t)row * a.in.chans + chb + lkB[q]);
        rb[q] = make_float4(activate(x.x, a.act), activate(x.y, a.act), activate(x.z, a.act),
                            activate(x.w, a.act));
      } else {
        rb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < A4; ++q) {
      As[buf][lkA[q] + 0][lrowA[q]] = ra[q].x;
      As[buf][lkA[q] + 1][lrowA[q]] = ra[q].y;
      As[buf][lkA[q] + 2][lrowA[q]] = ra[q].z;
      As[buf][lkA[q] + 3][lrowA[q]] = ra[q].w;
    }
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      Bs[buf][lkB[q] + 0][lrowB[q]] = rb[q].x;
      Bs[buf][lkB[q] + 1][lrowB[q]] = rb[q].y;
      Bs[buf][lkB[q] + 2][lrowB[q]] = rb[q].z;
      Bs[buf][lkB[q] + 3][lrowB[q]] = rb[q].w;
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  load(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int32_t kt = 0; kt < a.Kt; kt += BK) {
    const bool more = kt + BK < a.Kt;
    if (more) load(kt + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float am[TM], bn[TN];
#pragma unroll
      for (int g = 0; g < GM; ++g) {
        const float4 v = *reinterpret_cast<const float4*>(&As[buf][k][g * (BM / 2) + tx * 4]);
        am[g * 4 + 0] = v.x;
        am[g * 4 + 1] = v.y;
        am[g * 4 + 2] = v.z;
        am[g * 4 + 3] = v.w;
      }
#pragma unroll
      for (int g = 0; g < GN; ++g) {
        const float4 v = *reinterpret_cast<const float4*>(&Bs[buf][k][g * (BN / 2) + ty * 4]);
        bn[g * 4 + 0] = v.x;
        bn[g * 4 + 1] = v.y;
        bn[g * 4 + 2] = v.z;
        bn[g * 4 + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(am[i], bn[j], acc[i][j]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  int32_t ms[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) ms[i] = m0 + (i / 4) * (BM / 2) + tx * 4 + (i & 3);
  const bool vec = (a.cout % 4 == 0) && (a.M % 4 == 0);
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int32_t n = n0 + (j / 4) * (BN / 2) + ty * 4 + (j & 3);
    if (n >= N) continue;
    float col[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) col[i] = acc[i][j];
    store_column<TM>(a, n, ms, col, vec);
  }
}

// ---------------------------------------------------------------------------
// Narrow contraction (M <= 16 rows, Kt <= 64): four threads per
// GEMM column.  Thread q of a column's quad reduces indices 16q .. 16q+15 (its
// quarter of the window: four 16-byte loads when cin % 4 == 0, else one load
// per index) into all 16 rows; the quad then sums its partials with two XOR
// shuffles, in the fixed order (q0 + q1) + (q2 + q3), and thread q stores rows
// 4q .. 4q+3.  Used by the tail of the decoder (the noise branch's second
// conv, the inverse PQMF) and the encoder's PQMF analysis, whose launches are
// short chains of dependent work: four threads per column quarter each
// thread's chain.
// ---------------------------------------------------------------------------
constexpr int kSmallCols = 128;  // columns per block (threads = 4 x)
constexpr int kSmallRowPad = 4;  // floats of padding after every 16 reduction indices

__device__ __forceinline__ void small_column(const ConvArgs& a, bool valid, int32_t s, int32_t j, char* base,
                                             int32_t r0, const ColRows& cr, int q, const float* As) {
  const float* col = reinterpret_cast<const float*>(base + a.in.off) + a.in.choff;
  // this thread's quarter of the window, requested before any use: 16-byte
  // loads when cin % 4 == 0 (four consecutive indices never straddle a tap),
  // else one value per index (the PQMF analysis filterbank: cin = 1)
  const bool vec_in = a.cin % 4 == 0;
  float xw[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int32_t k = 16 * q + 4 * i;
    float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid && k < a.Kt) {
      if (vec_in) {
        const int32_t tap = k / a.cin, c = k - tap * a.cin;
        v4 = *reinterpret_cast<const float4*>(col + (int64_t)wrap_row(r0 + tap * a.dil, a.in.rows) * a.in.chans + c);
      } else {
        float e4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int32_t ke = k + e;
          const int32_t tap = ke / a.cin, c = ke - tap * a.cin;
          e4[e] = ke < a.Kt ? col[(int64_t)wrap_row(r0 + tap * a.dil, a.in.rows) * a.in.chans + c] : 0.f;
        }
        v4 = make_float4(e4[0], e4[1], e4[2], e4[3]);
      }
    }
    xw[4 * i] = activate(v4.x, a.act);
    xw[4 * i + 1] = activate(v4.y, a.act);
    xw[4 * i + 2] = activate(v4.z, a.act);
    xw[4 * i + 3] = activate(v4.w, a.act);
  }
  float acc[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) acc[m] = 0.f;
  // weights k-major, 16 rows per index, each quarter's block offset by
  // kSmallRowPad floats so the quad's four reads fall in distinct banks
  const float* Aq = As + q * (16 * 16 + kSmallRowPad);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float4* w4 = reinterpret_cast<const float4*>(Aq + i * 16);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float4 w = w4[g];
      acc[4 * g] = fmaf(w.x, xw[i], acc[4 * g]);
      acc[4 * g + 1] = fmaf(w.y, xw[i], acc[4 * g + 1]);
      acc[4 * g + 2] = fmaf(w.z, xw[i], acc[4 * g + 2]);
      acc[4 * g + 3] = fmaf(w.w, xw[i], acc[4 * g + 3]);
    }
  }
#pragma unroll
  for (int m = 0; m < 16; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 1);
#pragma unroll
  for (int m = 0; m < 16; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 2);
  if (!valid) return;  // a column past the batch (its quad's shuffles are done)
  float v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = q == 0 ? acc[i] : q == 1 ? acc[4 + i] : q == 2 ? acc[8 + i] : acc[12 + i];
  // an output that is only the caller's buffer with the 16 rows contiguous
  // there (one phase per row of one channel, or channels of one phase):
  // one 16-byte store per thread
  const bool ext_only = a.out.ext && !a.out.f32.rows && !a.out.lp[0].rows && !a.out.lp[1].rows && !a.has_skip;
  if (ext_only && a.M == 16 && (a.cout == 1 || a.phases == 1)) {
    float* e = a.out.ext + (int64_t)s * a.out.ext_stride + (int64_t)j * 16 + 4 * q;
    if ((reinterpret_cast<uintptr_t>(e) & 15) == 0) {
      float b4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) b4[i] = v[i] + (a.bias ? a.bias[a.cout == 1 ? 0 : 4 * q + i] : 0.f);
      *reinterpret_cast<float4*>(e) = make_float4(b4[0], b4[1], b4[2], b4[3]);
      return;
    }
  }
  const int32_t ms[4] = {4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3};
  store_column_rows<4>(a, s, j, base, cr, ms, v, (a.cout % 4 == 0) && (a.M % 4 == 0));
}

__global__ void __launch_bounds__(4 * kSmallCols, 2) k_conv_small_f32(const ConvArgs a) {
  // weights k-major ([Kt][16], rows past M zero; see small_column)
  __shared__ __align__(16) float As[4 * (16 * 16 + kSmallRowPad)];
  // Before the wait: the weights (written once at model creation), the
  // column's slot and step counter (final when any launch after the chain's
  // first starts: the slot list is uploaded before the chain; the counters
  // were advanced by the previous chain's last launch or, in this launch,
  // after every column has read them), and the ring rows that follow from
  // them (64-bit remainders, kept off the path after the wait)
  const int q = threadIdx.x & 3;
  const int32_t n = blockIdx.x * kSmallCols + (threadIdx.x >> 2);
  const int32_t N = a.batch.count * a.ncols;
  int32_t s = 0, j = 0, slot = 0, r0 = 0;
  ColRows cr{0, 0, 0, 0};
  if (n < N) {
    s = n / a.ncols;
    j = n - s * a.ncols;
    slot = a.batch.slots[s];
    const int64_t step = a.batch.counters[slot];
    r0 = (int32_t)ring_row(step * a.in.u + (int64_t)j * a.stride - a.hist, a.in.rows);
    cr = col_rows(a, step, j);
  }
  for (int i = threadIdx.x; i < 16 * 64; i += 4 * kSmallCols) {
    const int m = i & 15, k = i >> 4;
    As[(k >> 4) * (16 * 16 + kSmallRowPad) + (k & 15) * 16 + m] = (m < a.M && k < a.Kt) ? a.A[m * a.Kt + k] : 0.f;
  }
  __syncthreads();
  pdl_wait();
  pdl_release();
  // a column past the batch still takes part in its quad's shuffles
  small_column(a, n < N, s, j, a.batch.arena + (int64_t)slot * a.batch.slot_bytes, r0, cr, q, As);
  if (a.advance) {
    // the last launch of the chain: this block's columns are whole streams
    // (128 a multiple of the columns per stream, or equal to them); once every
    // thread has read its stream's counter, the block advances them
    __syncthreads();
    const int32_t s0 = blockIdx.x * kSmallCols / a.ncols;
    const int32_t s1 = min((blockIdx.x * kSmallCols + kSmallCols - 1) / a.ncols + 1, a.batch.count);
    if ((int32_t)threadIdx.x < s1 - s0)
      const_cast<int64_t*>(a.batch.counters)[a.batch.slots[s0 + threadIdx.x]] += a.advance;
  }
}


// ---------------------------------------------------------------------------
// Element-wise kernels
// ---------------------------------------------------------------------------
// Input-manipulation noise: the same uniform draw, from the generator whose
// seed is the stream seed XOR kInputNoiseTag (a domain apart from the heads'
// noise), counter = frame * channels + channel over input frames.
constexpr uint64_t kInputNoiseTag = 0x6C6174656E742D6Eull;
__device__ __forceinline__ float input_noise(uint64_t seed, int64_t frame, int32_t c, int32_t channels) {
  return noise_uniform(seed ^ kInputNoiseTag, frame, c, channels);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// One thread per (stream, frame, group of four bands): short chains of
// dependent work (three 16-byte branch loads, four tanh / sigmoid / noise
// evaluations, the view stores), four threads per frame of 16 bands.  What
// depends only on the stream's slot, step and seed (ring rows, addresses, the
// noise draws) is prepared before the dependency wait.
struct HeadsItem {
  const float* in[3];  // the three branches' values of bands b0 .. b0+3
  float* fo;           // FP32 view row (+ b0) or null
  float* eo;           // caller's buffer (+ b0) or null
  char* base;          // the stream's slot
  int32_t r0, r1;      // low-precision view rows
  int32_t b0;
  bool vec4;
  float nz[4];         // noise draws u(t, b) of the four bands (0 without noise)
};

__device__ __forceinline__ HeadsItem heads_prep(const HeadsArgs& a, int64_t it, int32_t G, int32_t slot,
                                                int64_t step, uint64_t seed) {
  HeadsItem h;
  const int64_t nj = it / G;
  h.b0 = 4 * (int32_t)(it - nj * G);
  const int32_t s = (int32_t)(nj / a.ncols);
  const int32_t j = (int32_t)(nj - (int64_t)s * a.ncols);
  const int64_t t = step * a.out_u + j;
  h.base = a.batch.arena + (int64_t)slot * a.batch.slot_bytes;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    h.in[q] = reinterpret_cast<const float*>(h.base + a.in[q].off) +
              ring_row(t - a.A[q], a.in[q].rows) * a.in[q].chans + a.in[q].choff + h.b0;
  h.fo = a.out.f32.rows ? reinterpret_cast<float*>(h.base + a.out.f32.off) +
                              ring_row(t, a.out.f32.rows) * a.out.f32.chans + h.b0
                        : nullptr;
  h.eo = a.out.ext ? a.out.ext + (int64_t)s * a.out.ext_stride + (int64_t)j * a.bands + h.b0 : nullptr;
  h.r0 = a.out.lp[0].rows ? (int32_t)ring_row(t, a.out.lp[0].rows) : 0;
  h.r1 = a.out.lp[1].rows ? (int32_t)ring_row(t, a.out.lp[1].rows) : 0;
  // 16-byte loads of the branches and store of the FP32 view when every
  // row is 16-byte aligned (channel counts and offsets multiples of 4)
  bool vec4 = (a.bands & 3) == 0 && (!h.fo || (reinterpret_cast<uintptr_t>(h.fo) & 15) == 0);
#pragma unroll
  for (int q = 0; q < 3; ++q) vec4 = vec4 && (reinterpret_cast<uintptr_t>(h.in[q]) & 15) == 0;
  h.vec4 = vec4;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int32_t b = h.b0 + e;
    h.nz[e] = (a.noise && b < a.bands) ? noise_uniform(seed, t - a.delay, b, a.bands) : 0.f;
  }
  return h;
}

__device__ __forceinline__ void heads_item(const HeadsArgs& a, const HeadsItem& h) {
  float v[3][4];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (h.vec4) {
      const float4 t4 = *reinterpret_cast<const float4*>(h.in[q]);
      v[q][0] = t4.x;
      v[q][1] = t4.y;
      v[q][2] = t4.z;
      v[q][3] = t4.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[q][e] = h.b0 + e < a.bands ? h.in[q][e] : 0.f;
    }
  }
  float y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    y[e] = tanhf(v[0][e]) * sigmoidf_(v[1][e]);
    if (a.noise && h.b0 + e < a.bands) y[e] += sigmoidf_(v[2][e]) * h.nz[e];
  }
  if (h.fo && h.vec4) {
    *reinterpret_cast<float4*>(h.fo) = make_float4(y[0], y[1], y[2], y[3]);
  } else if (h.fo) {
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (h.b0 + e < a.bands) h.fo[e] = y[e];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (h.b0 + e >= a.bands) break;
    if (h.eo) h.eo[e] = y[e];
    if (a.out.lp[0].rows) store_lp(h.base, a.out.lp[0], h.r0, h.b0 + e, y[e]);
    if (a.out.lp[1].rows) store_lp(h.base, a.out.lp[1], h.r1, h.b0 + e, leaky(y[e]));
  }
}

__global__ void k_heads(const HeadsArgs a) {
  const int32_t G = (a.bands + 3) / 4;  // band groups per frame
  const int64_t total = (int64_t)a.batch.count * a.ncols * G;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the first item prepared before the wait: its stream's slot, step counter
  // and seed are final when any launch after the chain's first starts (the
  // heads never start a chain)
  HeadsItem h0;
  if (i0 < total) {
    const int32_t slot = a.batch.slots[i0 / G / a.ncols];
    h0 = heads_prep(a, i0, G, slot, a.batch.counters[slot], a.batch.seeds[slot]);
  }
  pdl_wait();
  pdl_release();
  if (i0 < total) heads_item(a, h0);
  for (int64_t it = i0 + (int64_t)gridDim.x * blockDim.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = a.batch.slots[it / G / a.ncols];
    heads_item(a, heads_prep(a, it, G, slot, a.batch.counters[slot], a.batch.seeds[slot]));
  }
}

__global__ void k_add(const AddArgs a) {
  pdl_wait();
  pdl_release();
  const int32_t C = a.chans;
  const int64_t total = (int64_t)a.batch.count * a.ncols * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i % C);
    const int64_t nj = i / C;
    const int32_t j = (int32_t)(nj % a.ncols);
    const int32_t s = (int32_t)(nj / a.ncols);
    const int64_t t = steps_of(a.batch, s) * a.out_u + j;
    float y = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float* p = ring_ptr<const float>(a.batch, s, a.in[q]);
      y += p[ring_row(t - a.A[q], a.in[q].rows) * a.in[q].chans + a.in[q].choff + c];
    }
    store_views(a.batch, s, a.out, t, j, c, C, y);
  }
}

__global__ void k_input(const InputArgs a) {
  pdl_wait();
  pdl_release();
  const int32_t C = a.chans;
  const int64_t total = (int64_t)a.batch.count * a.ncols * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i % C);
    const int64_t nj = i / C;
    const int32_t j = (int32_t)(nj % a.ncols);
    const int32_t s = (int32_t)(nj / a.ncols);
    const int64_t t = steps_of(a.batch, s) * a.out_u + j;
    // the stream's input manipulation x' = scale * x + bias + amp * u(t, c)
    // (the identity 1, 0, 0 leaves x unchanged)
    const int32_t slot = a.batch.slots[s];
    const float* mp = a.manip + (int64_t)slot * 3 * C;
    const float x = a.src[(int64_t)s * a.src_stride + (int64_t)j * C + c];
    float v = fmaf(mp[c], x, mp[C + c]);
    const float amp = mp[2 * C + c];
    if (amp != 0.f) v = fmaf(amp, input_noise(a.batch.seeds[slot], t, c, C), v);
    store_views(a.batch, s, a.out, t, j, c, C, v);
  }
}

__global__ void k_advance(const Batch b, int64_t steps) {
  pdl_wait();
  pdl_release();
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < b.count) const_cast<int64_t*>(b.counters)[b.slots[s]] += steps;
}

int elementwise_grid(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

static bool takes_small(const ConvArgs& a) { return a.M <= 16 && a.Kt <= 64; }

bool conv_f32_can_advance(const ConvArgs& a) {
  return takes_small(a) && a.ncols > 0 && (a.ncols == kSmallCols || kSmallCols % a.ncols == 0);
}

cudaError_t launch_conv_f32(const ConvArgs& a, cudaStream_t st) {
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  if (N <= 0) return cudaSuccess;
  if (a.advance && !conv_f32_can_advance(a)) return cudaErrorInvalidValue;
  auto tiles = [&](int bm, int bn) { return ((a.M + bm - 1) / bm) * ((N + bn - 1) / bn); };
  if (takes_small(a)) {
    dim3 grid((unsigned)((N + kSmallCols - 1) / kSmallCols));
    return launch_pdl(k_conv_small_f32, grid, dim3(4 * kSmallCols), 0, st, a);
  }
  if (a.cin % 8 == 0 && a.M >= 128 && tiles(128, 128) >= 2 * 152) {
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((a.M + 127) / 128));
    return launch_pdl(k_conv_tile_f32<128, 128, 8>, grid, dim3(256), 0, st, a);
  } else if (a.cin % 16 == 0 && N >= 32) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((a.M + 63) / 64));
    return launch_pdl(k_conv_tile_f32<64, 64, 16>, grid, dim3(256), 0, st, a);
  } else {
    dim3 grid((unsigned)((N + kGemvCols - 1) / kGemvCols),
              (unsigned)((a.M + kGemvWarps - 1) / kGemvWarps));
    if (a.cin % 4 == 0 && a.cin >= 64)
      return launch_pdl(k_conv_gemv_f32<true>, grid, dim3(kGemvWarps * 32), 0, st, a);
    else
      return launch_pdl(k_conv_gemv_f32<false>, grid, dim3(kGemvWarps * 32), 0, st, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_heads(const HeadsArgs& a, cudaStream_t st) {
  // one thread per (stream, frame, group of four bands)
  const int64_t total = (int64_t)a.batch.count * a.ncols * ((a.bands + 3) / 4);
  if (total <= 0) return cudaSuccess;
  return launch_pdl(k_heads, dim3(elementwise_grid(total)), dim3(256), 0, st, a);
}

cudaError_t launch_add(const AddArgs& a, cudaStream_t st) {
  const int64_t total = (int64_t)a.batch.count * a.ncols * a.chans;
  if (total <= 0) return cudaSuccess;
  return launch_pdl(k_add, dim3(elementwise_grid(total)), dim3(256), 0, st, a);
}

cudaError_t launch_input(const InputArgs& a, cudaStream_t st) {
  const int64_t total = (int64_t)a.batch.count * a.ncols * a.chans;
  if (total <= 0) return cudaSuccess;
  return launch_pdl(k_input, dim3(elementwise_grid(total)), dim3(256), 0, st, a);
}

cudaError_t launch_advance(const Batch& b, int64_t steps, cudaStream_t st) {
  if (b.count <= 0) return cudaSuccess;
  return launch_pdl(k_advance, dim3((b.count + 255) / 256), dim3(256), 0, st, b, steps);
}

}  // namespace cc
