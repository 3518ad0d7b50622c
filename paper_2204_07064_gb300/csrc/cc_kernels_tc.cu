// Tensor-core (tcgen05) cached convolution for batched streams: the channel
// contraction of Eq. 1 (and of the polyphase transposed convolution) as an
// implicit GEMM  D[M][N] = A[M][taps*cin] . B[N][taps*cin]^T  where the N
// columns are (stream, frame) pairs and B row n, tap k is the ring-buffer row
// of that stream at time t0 + j*stride + k*dil - hist (cached padding,
// section 2.2, read in place).
//
// One CTA computes a 128 x BN tile:
//   warps 0-3  producers: TMA for the weight tile (128 rows x 64 K, 128-byte
//              swizzle), cp.async gathers of the BN window rows into the same
//              swizzled layout; then the epilogue (TMEM -> registers ->
//              scale, bias, aligned residual, every output view)
//   warp 4     TMEM allocation; lane 0 issues tcgen05.mma (128 x BN x 16,
//              BF16 or FP16 operands, FP32 accumulation in TMEM)
// Stages are handed over with mbarriers; every wait is bounded in time and
// records an error in the model's device error word instead of hanging.
#include <cuda.h>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_sm100.cuh"

namespace cc {
namespace {

using namespace sm100;

constexpr int kStages = 4;
constexpr int kBM = 128;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

template <int BN>
struct TcLayout {
  static constexpr int kA = kBM * 128;  // one 128 x 64 low-precision tile
  static constexpr int kB = BN * 128;
  static constexpr int kBars = (2 * kStages + 1) * 8 + 8;
  static constexpr int kCols = BN * (8 + 8 + 4 * 4);
  static constexpr int kBytes = 1024 + kStages * (kA + kB) + kBars + kCols + 64;
};

template <int BN>
__global__ void __launch_bounds__(160, 1) k_conv_tc(const __grid_constant__ CUtensorMap tmA,
                                                    const TcArgs a) {
  using L = TcLayout<BN>;
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
      mbar_init(full + s, 129);  // 128 gather arrivals + 1 expect_tx arrival
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull, 1);
    fence_mbar_init();
    prefetch_tmap(&tmA);
  }
  if (warp == 4) {
    tmem_alloc(tbase, BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;

  if (warp < 4) {
    const int t = threadIdx.x;
    // ---- per-column epilogue addressing (stream slot, output rows per view)
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
    // ---- producer: gather rows of the cached window
    constexpr int RPT = BN / 128;
    const uint16_t* bbase[RPT];
    int32_t br0[RPT];
    bool bok[RPT];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int64_t n = n0 + t + rr * 128;
      bok[rr] = n < N;
      bbase[rr] = nullptr;
      br0[rr] = 0;
      if (bok[rr]) {
        const int32_t s = (int32_t)(n / a.ncols);
        const int32_t j = (int32_t)(n - (int64_t)s * a.ncols);
        bbase[rr] = reinterpret_cast<const uint16_t*>(slot_base(a.batch, s) + a.in.off);
        const int64_t tin = steps_of(a.batch, s) * a.in.u + (int64_t)j * a.stride - a.hist;
        br0[rr] = (int32_t)ring_row(tin, a.in.rows);
      }
    }
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % kStages;
      const uint32_t ph = (kc / kStages) & 1;
      if (!mbar_wait(empty + st, ph ^ 1, kWaitNs)) {
        ok = false;
        break;
      }
      const int tap = kc / cchunks;
      const int c0 = (kc - tap * cchunks) * 64;
      if (t == 0) {
        mbar_arrive_expect_tx(full + st, L::kA);
        tma_load_2d(sA + st * L::kA, &tmA, full + st, kc * 64, m0);
      }
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        const int r = t + rr * 128;
        const uint16_t* src = reinterpret_cast<const uint16_t*>(a.scale);  // any valid address
        if (bok[rr]) {
          const int32_t row = wrap_row(br0[rr] + tap * a.dil, a.in.rows);
          src = bbase[rr] + (int64_t)row * a.cin + c0;
        }
        uint8_t* dst = sB + st * L::kB;
#pragma unroll
        for (int c = 0; c < 8; ++c) cp_async_16(dst + sw128_offset(r, c), src + c * 8, bok[rr] ? 16u : 0u);
      }
      cp_async_commit();
      if (kc > 0) {
        cp_async_wait<1>();
        fence_proxy_async_smem();
        mbar_arrive(full + (kc - 1) % kStages);
      }
    }
    cp_async_wait<0>();
    fence_proxy_async_smem();
    if (ok && nk > 0) mbar_arrive(full + (nk - 1) % kStages);
    if (!ok) atomicOr(a.err, 1);

    // ---- epilogue
    asm volatile("bar.sync 1, 128;" ::: "memory");  // column table written by all producers
    bool got = mbar_wait(tfull, 0, kWaitNs);
    got = __all_sync(0xffffffffu, got);
    tc_fence_after();
    if (!got) {
      if (lane == 0) atomicOr(a.err, 2);
    } else {
      const int32_t m = m0 + warp * 32 + lane;
      const bool mok = m < a.M;
      int32_t ph = 0, ch = m;
      if (a.phases > 1) {
        ph = m / a.cout;
        ch = m - ph * a.cout;
      }
      const float sc = mok ? a.scale[m] : 0.f;
      const float bi = (mok && a.bias) ? a.bias[ch] : 0.f;
      for (int cb = 0; cb < BN; cb += 32) {
        if (n0 + cb >= N) break;
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
        tmem_ld_wait();
        if (!mok) continue;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int c = cb + jj;
          if (n0 + c >= N) continue;
          float v = __uint_as_float(r[jj]) * sc + bi;
          char* base = a.batch.arena + col_slot[c];
          if (a.has_skip) {
            const int32_t row = wrap_row(col_row[3 * BN + c] + ph, a.skip.rows);
            v += reinterpret_cast<const float*>(base + a.skip.off)[(int64_t)row * a.skip.chans + ch];
          }
          if (a.out.ext) a.out.ext[col_ext[c] + (int64_t)ph * a.cout + ch] = v;
          if (a.out.f32.rows) {
            const int32_t row = wrap_row(col_row[c] + ph, a.out.f32.rows);
            reinterpret_cast<float*>(base + a.out.f32.off)[(int64_t)row * a.out.f32.chans + ch] = v;
          }
          if (a.out.lp[0].rows)
            store_lp(base, a.out.lp[0], wrap_row(col_row[BN + c] + ph, a.out.lp[0].rows), ch, v);
          if (a.out.lp[1].rows)
            store_lp(base, a.out.lp[1], wrap_row(col_row[2 * BN + c] + ph, a.out.lp[1].rows), ch,
                     leaky(v));
        }
      }
    }
  } else if (warp == 4 && lane == 0) {
    // ---- MMA issuer
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
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 4) tmem_dealloc(tmem, BN);
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap& tm, const TcArgs& a, cudaStream_t st) {
  static bool configured = false;
  constexpr int bytes = TcLayout<BN>::kBytes;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  const int mtiles = (a.M + kBM - 1) / kBM;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)mtiles);
  k_conv_tc<BN><<<grid, 160, bytes, st>>>(tm, a);
  return cudaGetLastError();
}

}  // namespace

int tc_tile_n(int64_t n_cols, int m_tiles) {
  return ((n_cols + 255) / 256) * m_tiles >= 152 ? 256 : 128;
}

cudaError_t launch_conv_tc(const void* tmap, const TcArgs& a, int bn, cudaStream_t st) {
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  if (N <= 0) return cudaSuccess;
  const CUtensorMap& tm = *reinterpret_cast<const CUtensorMap*>(tmap);
  return bn == 256 ? launch_bn<256>(tm, a, st) : launch_bn<128>(tm, a, st);
}

}  // namespace cc
