// Tensor-core (tcgen05) cached convolution for batched streams: the channel
// contraction of Eq. 1 (and of the polyphase transposed convolution) as an
// implicit GEMM  D[M][N] = A[M][taps*cin] . B[N][taps*cin]^T  where the N
// columns are (stream, frame) pairs and B row n, tap k is the ring-buffer row
// of that stream at time t0 + j*stride + k*dil - hist (cached padding,
// section 2.2, read in place).
//
// One CTA computes a 128 x BN tile with three roles:
//   warp 0     TMA producer: per 64-wide K slice, the weight tile (stored
//              pre-tiled and pre-swizzled, so one 16 KB bulk copy) and the BN
//              window rows, gathered four at a time (tile::gather4) from the
//              stream rings into the 128-byte-swizzled operand layout; one
//              expect-tx per stage, no thread waits on its own copies, so
//              every stage can be in flight
//   warp 1     TMEM allocation; lane 0 issues tcgen05.mma (128 x BN x 16,
//              BF16 or FP16 operands, FP32 accumulation in TMEM)
//   warps 2-5  epilogue: TMEM -> registers -> transposed shared memory ->
//              scale, bias, aligned residual, 16/32-byte stores of every view
// Every mbarrier wait is bounded in time and records an error in the model's
// device error word instead of hanging.
#include <cuda.h>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_sm100.cuh"

namespace cc {
namespace {

using namespace sm100;

constexpr int kBM = 128;
constexpr int kThreads = 192;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

// Pipeline depth: 128-column tiles run with 2 stages (three CTAs per SM, so
// the CTAs' epilogues overlap each other's main loops; deeper pipelines with
// fewer CTAs measured no faster); 256-column tiles use 4 stages, one CTA per SM.
template <int BN, int STAGES>
struct TcLayout {
  static constexpr int kStages = STAGES;
  static constexpr int kA = kBM * 128;  // one 128 x 64 low-precision tile
  static constexpr int kB = BN * 128;
  static constexpr int kBars = (2 * kStages + 1) * 8 + 8;
  static constexpr int kCols = BN * (8 + 8 + 4 * 4);
  static constexpr int kBytes = 1024 + kStages * (kA + kB) + kBars + kCols + 64;
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, STAGES == 2 ? 3 : 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const TcArgs a) {
  using L = TcLayout<BN, STAGES>;
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * L::kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * L::kB);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint32_t* tbase = reinterpret_cast<uint32_t*>(tfull + 1);
  int64_t* col_slot = reinterpret_cast<int64_t*>(tbase + 2);
  int64_t* col_ext = col_slot + BN;
  int32_t* col_row = reinterpret_cast<int32_t*>(col_ext + BN);  // [4][BN]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t m0 = blockIdx.y * kBM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  const int nk = a.Kt / 64;
  const int cchunks = a.cin / 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);  // the producer's expect-tx arrival; TMA completes the bytes
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull, 1);
    fence_mbar_init();
    prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(tbase, BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // The weight tiles of the first stages do not depend on earlier kernels:
    // they are requested before waiting for the previous layer.
    const int pre = nk < kStages ? nk : kStages;
    const uint8_t* atile = static_cast<const uint8_t*>(a.A_tiled) + (size_t)blockIdx.y * nk * L::kA;
    if (lane == 0)
      for (int kc = 0; kc < pre; ++kc) {
        mbar_arrive_expect_tx(full + kc, L::kA + L::kB);
        bulk_load(sA + kc * L::kA, atile + (size_t)kc * L::kA, L::kA, full + kc);
      }
    pdl_wait();
    pdl_release();
    // lane l gathers tile rows 4*(l + 32*g) .. +3 for g < BN/128
    constexpr int G = BN / 128;
    int32_t ybase[G][4], r0[G][4];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t n = n0 + 4 * (lane + 32 * g) + i;
        ybase[g][i] = 0;
        r0[g][i] = -1;  // column past the batch: read arena row 0, result discarded
        if (n < N) {
          const int32_t s = (int32_t)(n / a.ncols);
          const int32_t j = (int32_t)(n - (int64_t)s * a.ncols);
          ybase[g][i] = a.batch.slots[s] * a.in_rows_per_slot + a.in_row_off;
          r0[g][i] = (int32_t)ring_row(steps_of(a.batch, s) * a.in.u + (int64_t)j * a.stride - a.hist,
                                       a.in.rows);
        }
      }
    bool ok = true;
    int issued = 0;
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % kStages;
      const uint32_t ph = (kc / kStages) & 1;
      if (!mbar_wait(empty + st, ph ^ 1, kWaitNs)) {
        ok = false;
        break;
      }
      const int tap = kc / cchunks;
      const int c0 = (kc - tap * cchunks) * 64;
      if (lane == 0 && kc >= pre) {
        mbar_arrive_expect_tx(full + st, L::kA + L::kB);
        bulk_load(sA + st * L::kA, atile + (size_t)kc * L::kA, L::kA, full + st);
      }
      __syncwarp();
      uint8_t* dst = sB + st * L::kB;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        int32_t y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          y[i] = r0[g][i] < 0 ? 0 : ybase[g][i] + wrap_row(r0[g][i] + tap * a.dil, a.in.rows);
        tma_gather4(dst + (lane + 32 * g) * 512, &tmB, full + st, c0, y[0], y[1], y[2], y[3]);
      }
      issued = kc + 1;
    }
    if (!ok) {
      if (lane == 0) atomicOr(a.err, 1);
      // let the copies already issued land before the CTA's shared memory goes away
      for (int kc = issued - kStages < 0 ? 0 : issued - kStages; kc < issued; ++kc)
        mbar_wait(full + kc % kStages, (kc / kStages) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    pdl_wait();
    pdl_release();
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(kBM, BN, a.in.dtype == kDtBF16);
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % kStages;
        const uint32_t ph = (kc / kStages) & 1;
        if (!mbar_wait(full + st, ph, kWaitNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(sA + st * L::kA), sb = smem_u32(sB + st * L::kB);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_f16(tmem, sw128_kmajor_desc(sa + k * 32), sw128_kmajor_desc(sb + k * 32), idesc,
                  (kc | k) != 0);
        mma_commit(empty + st);
      }
      mma_commit(tfull);
      if (!ok) atomicOr(a.err, 4);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int t = threadIdx.x - 64;  // 0..127
    const int sub = warp & 3;        // TMEM lane quarter this warp may access
    pdl_wait();
    pdl_release();
    for (int c = t; c < BN; c += 128) {
      const int64_t n = n0 + c;
      if (n < N) {
        const int32_t s = (int32_t)(n / a.ncols);
        const int32_t j = (int32_t)(n - (int64_t)s * a.ncols);
        col_slot[c] = (int64_t)a.batch.slots[s] * a.batch.slot_bytes;
        col_ext[c] = (int64_t)s * a.out.ext_stride + (int64_t)j * a.phases * a.cout;
        const int64_t tb = steps_of(a.batch, s) * a.out_u + (int64_t)j * a.phases;
        col_row[0 * BN + c] = a.out.f32.rows ? (int32_t)ring_row(tb, a.out.f32.rows) : 0;
        col_row[1 * BN + c] = a.out.lp[0].rows ? (int32_t)ring_row(tb, a.out.lp[0].rows) : 0;
        col_row[2 * BN + c] = a.out.lp[1].rows ? (int32_t)ring_row(tb, a.out.lp[1].rows) : 0;
        col_row[3 * BN + c] = a.has_skip ? (int32_t)ring_row(tb - a.skip_A, a.skip.rows) : 0;
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // column table complete
    // Residual values of pass 2 (below), software-pipelined one 32-column
    // chunk ahead: chunk 0's are requested before the accumulator is ready.
    float4 skip_next[4][2];
    auto fetch_skip = [&](int cb, float4 (&dst)[4][2]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = t + q * 128;
        const int c = p >> 4, g = p & 15;
        const int32_t mb = m0 + g * 8;
        dst[q][0] = dst[q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!a.has_skip || cb >= BN || n0 + cb + c >= N || mb >= a.M) continue;
        const int32_t ph = a.phases > 1 ? mb / a.cout : 0;
        const int32_t cg = mb - ph * a.cout;
        const int col = cb + c;
        const int32_t row = wrap_row(col_row[3 * BN + col] + ph, a.skip.rows);
        const float4* sp = reinterpret_cast<const float4*>(a.batch.arena + col_slot[col] + a.skip.off +
                                                           ((int64_t)row * a.skip.chans + cg) * 4);
        dst[q][0] = __ldg(sp);
        dst[q][1] = __ldg(sp + 1);
      }
    };
    fetch_skip(0, skip_next);
    // one verdict for all 128 epilogue threads (a reduction barrier), so the
    // named barriers below always match
    const bool waited = mbar_wait(tfull, 0, kWaitNs);
    uint32_t all_ok;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(all_ok)
        : "r"((uint32_t)waited)
        : "memory");
    tc_fence_after();
    if (!all_ok) {
      if (t == 0) atomicOr(a.err, 2);
    } else {
      // Two passes per 32-column TMEM chunk.  Pass 1: thread = output row,
      // scaled + biased values go transposed into shared memory (the free
      // pipeline buffers).  Pass 2: thread = (column, 8 consecutive rows):
      // 16/32-byte residual loads and view stores, coalesced along channels.
      const int32_t rloc = sub * 32 + lane;
      const int32_t m = m0 + rloc;
      const bool mok = m < a.M;
      int32_t ch = m;
      if (a.phases > 1) ch = m - (m / a.cout) * a.cout;
      const float sc = mok ? a.scale[m] : 0.f;
      const float bi = (mok && a.bias) ? a.bias[ch] : 0.f;
      float* stage = reinterpret_cast<float*>(sA);  // 2 x 32 x 128 floats
      for (int cb = 0, it = 0; cb < BN; cb += 32, ++it) {
        if (n0 + cb >= N) break;  // uniform over the 128 epilogue threads
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)cb, r);
        tmem_ld_wait();
        float* stg = stage + (it & 1) * 32 * kBM;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) stg[jj * kBM + rloc] = __uint_as_float(r[jj]) * sc + bi;
        float4 skip_cur[4][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          skip_cur[q][0] = skip_next[q][0];
          skip_cur[q][1] = skip_next[q][1];
        }
        fetch_skip(cb + 32, skip_next);
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int p = t + q * 128;
          const int c = p >> 4, g = p & 15;
          const int32_t mb = m0 + g * 8;
          if (n0 + cb + c >= N || mb >= a.M) continue;
          float x[8];
          const float4 x0 = *reinterpret_cast<const float4*>(stg + c * kBM + g * 8);
          const float4 x1 = *reinterpret_cast<const float4*>(stg + c * kBM + g * 8 + 4);
          x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
          x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
          const int32_t ph = a.phases > 1 ? mb / a.cout : 0;
          const int32_t cg = mb - ph * a.cout;  // first channel of the group
          const int col = cb + c;
          char* base = a.batch.arena + col_slot[col];
          if (a.has_skip) {
            const float4 s0 = skip_cur[q][0], s1 = skip_cur[q][1];
            x[0] += s0.x; x[1] += s0.y; x[2] += s0.z; x[3] += s0.w;
            x[4] += s1.x; x[5] += s1.y; x[6] += s1.z; x[7] += s1.w;
          }
          if (a.out.ext) {
            float* e = a.out.ext + col_ext[col] + (int64_t)ph * a.cout + cg;
#pragma unroll
            for (int k = 0; k < 8; ++k) e[k] = x[k];
          }
          if (a.out.f32.rows) {
            const int32_t row = wrap_row(col_row[col] + ph, a.out.f32.rows);
            float4* d = reinterpret_cast<float4*>(base + a.out.f32.off +
                                                  ((int64_t)row * a.out.f32.chans + cg) * 4);
            d[0] = make_float4(x[0], x[1], x[2], x[3]);
            d[1] = make_float4(x[4], x[5], x[6], x[7]);
          }
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const Ring& lr = a.out.lp[v];
            if (!lr.rows) continue;
            const int32_t row = wrap_row(col_row[(1 + v) * BN + col] + ph, lr.rows);
            float y[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) y[k] = v ? leaky(x[k]) : x[k];
            uint4 pk;
            if (lr.dtype == kDtBF16) {
              __nv_bfloat162 h0 = __floats2bfloat162_rn(y[0], y[1]), h1 = __floats2bfloat162_rn(y[2], y[3]);
              __nv_bfloat162 h2 = __floats2bfloat162_rn(y[4], y[5]), h3 = __floats2bfloat162_rn(y[6], y[7]);
              pk.x = *reinterpret_cast<uint32_t*>(&h0); pk.y = *reinterpret_cast<uint32_t*>(&h1);
              pk.z = *reinterpret_cast<uint32_t*>(&h2); pk.w = *reinterpret_cast<uint32_t*>(&h3);
            } else {
              __half2 h0 = __floats2half2_rn(y[0], y[1]), h1 = __floats2half2_rn(y[2], y[3]);
              __half2 h2 = __floats2half2_rn(y[4], y[5]), h3 = __floats2half2_rn(y[6], y[7]);
              pk.x = *reinterpret_cast<uint32_t*>(&h0); pk.y = *reinterpret_cast<uint32_t*>(&h1);
              pk.z = *reinterpret_cast<uint32_t*>(&h2); pk.w = *reinterpret_cast<uint32_t*>(&h3);
            }
            *reinterpret_cast<uint4*>(base + lr.off + ((int64_t)row * lr.chans + cg) * 2) = pk;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, BN);
}

template <int BN, int STAGES>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, cudaStream_t st) {
  static bool configured = false;
  constexpr int bytes = TcLayout<BN, STAGES>::kBytes;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_conv_tc<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  const int mtiles = (a.M + kBM - 1) / kBM;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)mtiles);
  return launch_pdl(k_conv_tc<BN, STAGES>, grid, dim3(kThreads), (size_t)bytes, st, ta, tb, a);
}

}  // namespace

int tc_tile_n(int64_t n_cols, int m_tiles) {
  return ((n_cols + 255) / 256) * m_tiles >= 152 ? 256 : 128;
}

cudaError_t launch_conv_tc(const void* tmap_a, const void* tmap_b, const TcArgs& a, int bn,
                           cudaStream_t st) {
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  if (N <= 0) return cudaSuccess;
  const CUtensorMap& ta = *reinterpret_cast<const CUtensorMap*>(tmap_a);
  const CUtensorMap& tb = *reinterpret_cast<const CUtensorMap*>(tmap_b);
  if (bn == 256) return launch_bn<256, 4>(ta, tb, a, st);
  return launch_bn<128, 2>(ta, tb, a, st);
}

}  // namespace cc
