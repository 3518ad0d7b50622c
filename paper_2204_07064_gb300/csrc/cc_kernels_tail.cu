// The stream-local tail of a launch chain as one persistent kernel.
//
// Late layers of a streamed model read only their own stream's frames: a
// cached convolution reads its window (this call's frames and the cached
// history, section 2.2) from its stream's rings, a transposed convolution its
// stream's input frames, a merge its stream's branches (Eq. 3).  So the suffix
// of the launch chain whose layers are all small enough to be run by one CTA
// needs no grid-wide synchronisation between layers: each CTA owns a group of
// streams and runs every tail layer on them, one after another, with only
// CTA-local barriers in between.  This replaces one launch per layer (and the
// step-counter advance) by a single launch.
//
// Contractions use tcgen05 in transposed form: the MMA's M side is 128
// columns (stream, frame) of the layer, its N side the layer's output rows
// (channels, or phase x channel for a polyphase transposed convolution),
// D^T[col][row] = window[col][K] . W[row][K]^T.  The operands are the same
// 128-byte-swizzled K-major tiles as the batched kernel's (the window rows
// loaded by TMA, the pre-tiled weight blocks by bulk copies), with their roles
// swapped in the descriptors.  TMEM lane = column, TMEM column = output row, so
// an epilogue thread owns one column and holds consecutive channels of it:
// its ring rows are written with 16-byte stores and no transpose, and a
// narrow layer (48 or 64 channels) takes an MMA of N = 48 or 64 instead of a
// half-empty 128-row tile.  A residual unit (k-wide conv -> 1x1 conv -> + skip)
// runs as one op: the first result, scaled, biased, activated and rounded, is
// written by the epilogue straight into shared memory as the second MMA's
// K-major A operand (each thread writes its own 128-byte row).
//
// Roles: warp 0 producer (weights by bulk copy, window rows by 3D TMA boxes,
// one box per stream run of a tile, or tile::gather4 row gathers when a run
// crosses its ring's end); warp 1 MMA issuer (lane 0) and TMEM owner; warps
// 2..9 epilogue (warp w reads TMEM lane quarter w % 4, i.e. 32 columns, and
// half (w - 2) / 4 of the rows).  The epilogue also runs the layers that are
// not contractions on tensor cores (narrow FP32 convolutions such as the
// inverse PQMF, the heads merge, unfused residual adds) as plain SIMT loops
// over the group's columns.
//
// Ordering inside a CTA: after each op every epilogue thread fences its global
// stores against the async proxy, the epilogue warps meet at a named barrier
// and one thread publishes the count of completed ops (release); the producer
// reads it (acquire) before it requests the next op's window rows (weights
// may already be in flight).  Two
// TMEM accumulator buffers let a tile's epilogue overlap the next tile's
// MMAs.  Every wait is bounded (wait_ns); a wait that gives up records its role
// in the model's error word, and every role then skips its remaining work.
#include <cuda.h>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_sm100.cuh"

namespace cc {
namespace {

using namespace sm100;

constexpr int kTailStages = 4;
constexpr int kTailEpiWarps = 8;
constexpr int kTailThreads = 64 + 32 * kTailEpiWarps;
constexpr int kTailEpi = 32 * kTailEpiWarps;
constexpr int kTile = 16384;  // 128 rows x 128 bytes
// shared memory: stages of (weight block, window tile), the fused unit's A
// operand (128 columns x 128 channels), barriers
constexpr int kTailSmem = 1024 + kTailStages * 2 * kTile + 2 * kTile + 256;

__device__ __forceinline__ bool bar_red_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kTailEpi)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTailEpi) : "memory"); }

// Completed-op counter in shared memory: the epilogue publishes with a
// release store after its warps met, the producer reads with acquire.
__device__ __forceinline__ void st_release_smem(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_smem(uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
// Waits until *p >= want; gives up after timeout_ns.
__device__ __forceinline__ bool wait_count(uint32_t* p, uint32_t want, uint64_t timeout_ns) {
  if (ld_acquire_smem(p) >= want) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t i = 1;; ++i) {
    if (ld_acquire_smem(p) >= want) return true;
    if ((i & 255u) == 0 && global_timer_ns() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// 32 lanes x 16 consecutive 32-bit TMEM columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ uint32_t pack_lp(float lo, float hi, bool bf16) {
  if (bf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// Per-op work of one group: its columns are (stream s, frame j) with s in
// [0, gs) of the group, j in [0, ncols), in stream-major order; tiles of 128.
struct GroupCols {
  int32_t s0, gs, ncols, tiles;
};

__device__ __forceinline__ GroupCols group_cols(const TailOp& op, const TailArgs& a, int32_t s0, int32_t gs) {
  GroupCols g;
  g.s0 = s0;
  g.gs = gs;
  g.ncols = op.u_cols * a.steps;
  g.tiles = (gs * g.ncols + 127) / 128;
  return g;
}

// Writes value v of output row (phase ph, channel ch) for column j of batch
// stream s (frames counted from the call's first) into every view of op.out
// and, for the last op, the caller's buffer.
__device__ __forceinline__ void put_value(const TailOp& op, const TailArgs& a, int32_t s, int64_t tb,
                                          int64_t local, int32_t ch, float v) {
  char* base = slot_base(a.batch, s);
  if (op.is_last) a.ext[(int64_t)s * a.ext_stride + local * op.cout + ch] = v;
  const Ring& f = op.out.f32;
  if (f.rows) reinterpret_cast<float*>(base + f.off)[ring_row(tb, f.rows) * f.chans + f.choff + ch] = v;
  if (op.out.lp[0].rows) store_lp(base, op.out.lp[0], ring_row(tb, op.out.lp[0].rows), ch, v);
  if (op.out.lp[1].rows) store_lp(base, op.out.lp[1], ring_row(tb, op.out.lp[1].rows), ch, leaky(v));
}

__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sW = smem;                                // [stages] weight blocks
  uint8_t* sX = smem + kTailStages * kTile;          // [stages] window tiles
  uint8_t* sU = smem + 2 * kTailStages * kTile;      // fused unit operand: 2 K slices
  uint64_t* full = reinterpret_cast<uint64_t*>(sU + 2 * kTile);
  uint64_t* empty = full + kTailStages;
  uint64_t* tfull = empty + kTailStages;  // [2]
  uint64_t* tfull2 = tfull + 2;           // [2]
  uint64_t* tempty = tfull2 + 2;          // [2]
  uint64_t* b2ready = tempty + 2;
  uint32_t* tbase = reinterpret_cast<uint32_t*>(b2ready + 1);
  volatile int32_t* abort_flag = reinterpret_cast<volatile int32_t*>(tbase + 1);
  uint32_t* ops_completed = tbase + 2;  // ops the epilogue has finished, all groups

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t n_groups = (a.batch.count + a.group - 1) / a.group;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTailStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tfull2 + b, 1);
      mbar_init(tempty + b, 1);
    }
    mbar_init(b2ready, 1);
    *abort_flag = 0;
    *ops_completed = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tbase, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  // every op may read what earlier launches of the chain wrote
  pdl_wait();
  pdl_release();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t slice = 0;    // running K-slice counter (stage, phase)
    uint32_t op_inst = 0;  // running op instance counter (every op of every group)
    bool ok = true;
    for (int32_t g = blockIdx.x; ok && g < n_groups; g += gridDim.x) {
      const int32_t s0 = g * a.group, gs = min(a.group, a.batch.count - s0);
      for (int32_t k = 0; ok && k < a.n_ops; ++k, ++op_inst) {
        const TailOp& op = a.ops[k];
        if (op.kind != kTailTc) continue;
        const GroupCols gc = group_cols(op, a, s0, gs);
        const CUtensorMap* maps = a.maps + (size_t)k * 9;
        const int cchunks = op.cin / 64;
        bool waited_dep = (k == 0);  // the group's first op reads earlier launches only
        for (int32_t t = 0; ok && t < gc.tiles; ++t) {
          // the tile's runs: boxes of one stream's consecutive frames when every
          // run is a power of two of rows and none crosses its ring's end
          const int32_t c0 = t * 128, c1 = min(c0 + 128, gs * gc.ncols);
          bool boxes = true;
          for (int32_t c = c0; c < c1;) {
            const int32_t s = c / gc.ncols, j = c - s * gc.ncols;
            const int32_t run = min(gc.ncols - j, c1 - c);
            const int64_t p = ring_row(steps_of(a.batch, s0 + s) * op.in.u, op.in.rows);
            if ((run & (run - 1)) != 0 || p + j + run > op.in.rows || (c - c0) % run != 0) boxes = false;
            c += run;
          }
          // bytes of the window tile: the boxes' rows, or all 128 gathered rows
          const uint32_t win_bytes = boxes ? (uint32_t)(c1 - c0) * 128u : (uint32_t)kTile;
          const int nslices = op.nk + op.k2;
          for (int i = 0; i < nslices; ++i, ++slice) {
            const int st = slice % kTailStages;
            const uint32_t ph = (slice / kTailStages) & 1;
            if (*abort_flag || !mbar_wait(empty + st, ph ^ 1, a.wait_ns)) {
              ok = false;
              break;
            }
            const bool window = i < op.nk;
            if (lane == 0) {
              mbar_arrive_expect_tx(full + st, window ? kTile + win_bytes : kTile);
              const uint8_t* wsrc = window ? static_cast<const uint8_t*>(op.A_tiled) + (size_t)i * kTile
                                           : static_cast<const uint8_t*>(op.A2_tiled) + (size_t)(i - op.nk) * kTile;
              bulk_load(sW + st * kTile, wsrc, kTile, full + st);
            }
            __syncwarp();
            if (!window) continue;
            if (!waited_dep) {
              // this op's window rows were written by earlier ops of the group:
              // wait until every op before this one has completed
              if (!wait_count(ops_completed, op_inst, a.wait_ns)) {
                ok = false;
                // the slice's expected bytes never come: its waiters give up too
                break;
              }
              fence_proxy_async_global();
              waited_dep = true;
            }
            const int tap = i / cchunks;
            const int ch0 = (i - tap * cchunks) * 64;
            uint8_t* dst = sX + st * kTile;
            if (boxes) {
              if (lane == 0) {
                for (int32_t c = c0; c < c1;) {
                  const int32_t s = c / gc.ncols, j = c - s * gc.ncols;
                  const int32_t run = min(gc.ncols - j, c1 - c);
                  int li = 0;
                  while ((1 << li) < run) ++li;
                  const int64_t p = ring_row(steps_of(a.batch, s0 + s) * op.in.u, op.in.rows);
                  const int32_t y = op.in.pre + (int32_t)p - op.hist + j + tap * op.dil;
                  tma_load_3d(dst + (c - c0) * 128, maps + li, full + st, ch0, y, a.batch.slots[s0 + s]);
                  c += run;
                }
                // rows of a partial tile past the group's columns stay as they
                // are: their results are never stored, and the tile's expected
                // bytes count only what is loaded
              }
            } else {
              // rows 4l .. 4l+3 of the tile per lane; rows past the group's
              // columns gather arena row 0 (results discarded)
              int32_t y[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int32_t c = c0 + 4 * lane + q;
                y[q] = 0;
                if (c < c1) {
                  const int32_t s = c / gc.ncols, j = c - s * gc.ncols;
                  const int64_t r0 =
                      ring_row(steps_of(a.batch, s0 + s) * op.in.u + j - op.hist + tap * op.dil, op.in.rows);
                  y[q] = a.batch.slots[s0 + s] * op.in_rows_per_slot + op.in_row_off + (int32_t)r0;
                }
              }
              tma_gather4(dst + lane * 512, maps + 8, full + st, ch0, y[0], y[1], y[2], y[3]);
            }
          }
        }
      }
    }
    if (!ok) *abort_flag = 1;
    // every issued copy lands before the CTA's shared memory goes away
    const uint32_t first = slice > (uint32_t)kTailStages ? slice - kTailStages : 0;
    bool drained = true;
    for (uint32_t i = first; i < slice; ++i)
      drained = mbar_wait(full + i % kTailStages, (i / kTailStages) & 1, a.wait_ns) && drained;
    if ((!ok || !drained) && lane == 0) atomicOr(a.err, 1);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t slice = 0, tile_j = 0, fused_j = 0;
      bool ok = true;
      for (int32_t g = blockIdx.x; ok && g < n_groups; g += gridDim.x) {
        const int32_t s0 = g * a.group, gs = min(a.group, a.batch.count - s0);
        for (int32_t k = 0; ok && k < a.n_ops; ++k) {
          const TailOp& op = a.ops[k];
          if (op.kind != kTailTc) continue;
          const GroupCols gc = group_cols(op, a, s0, gs);
          const uint32_t idesc = idesc_f16(128, op.N, op.lp_bf16 != 0);
          const uint32_t idesc2 = idesc_f16(128, op.N2 > 0 ? op.N2 : 16, op.lp_bf16 != 0);
          for (int32_t t = 0; ok && t < gc.tiles; ++t, ++tile_j) {
            const uint32_t buf = tile_j & 1;
            if (*abort_flag || !mbar_wait(tempty + buf, ((tile_j >> 1) & 1) ^ 1, a.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d1 = tmem + buf * 256;
            for (int i = 0; i < op.nk; ++i, ++slice) {
              const int st = slice % kTailStages;
              if (!mbar_wait(full + st, (slice / kTailStages) & 1, a.wait_ns)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sx = smem_u32(sX + st * kTile), sw = smem_u32(sW + st * kTile);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_f16(d1, sw128_kmajor_desc(sx + kk * 32), sw128_kmajor_desc(sw + kk * 32), idesc,
                        (i | kk) != 0);
              mma_commit(empty + st);
            }
            mma_commit(tfull + buf);
            if (!ok) break;
            if (op.k2 > 0) {
              // fused unit: the epilogue's operand, then the 1x1 conv into d1 + 128
              if (!mbar_wait(b2ready, fused_j & 1, a.wait_ns)) {
                ok = false;
                break;
              }
              ++fused_j;
              tc_fence_after();
              for (int i = 0; i < op.k2; ++i, ++slice) {
                const int st = slice % kTailStages;
                if (!mbar_wait(full + st, (slice / kTailStages) & 1, a.wait_ns)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t su = smem_u32(sU + i * kTile), sw = smem_u32(sW + st * kTile);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_f16(d1 + 128, sw128_kmajor_desc(su + kk * 32), sw128_kmajor_desc(sw + kk * 32), idesc2,
                          (i | kk) != 0);
                mma_commit(empty + st);
              }
              mma_commit(tfull2 + buf);
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 4);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int t = threadIdx.x - 64;      // 0 .. 255
    const int quarter = warp & 3;        // TMEM lane quarter
    const int half = (warp - 2) >> 2;    // which half of the output rows
    const int r = quarter * 32 + lane;   // this thread's column within a tile
    uint32_t tile_j = 0, op_count = 0;
    uint32_t fused_use[2] = {0, 0};  // fused tiles so far per accumulator buffer (tfull2 phases)
    bool ok = true;
    for (int32_t g = blockIdx.x; ok && g < n_groups; g += gridDim.x) {
      const int32_t s0 = g * a.group, gs = min(a.group, a.batch.count - s0);
      for (int32_t k = 0; ok && k < a.n_ops; ++k) {
        const TailOp& op = a.ops[k];
        const GroupCols gc = group_cols(op, a, s0, gs);
        const int32_t ncol_g = gs * gc.ncols;
        if (op.kind == kTailTc) {
          const bool lp_bf16 = op.lp_bf16 != 0;
          for (int32_t tt = 0; tt < gc.tiles; ++tt, ++tile_j) {
            const uint32_t buf = tile_j & 1;
            const int32_t c = tt * 128 + r;
            const bool cok = c < ncol_g;
            const int32_t sl = cok ? c / gc.ncols : 0;
            const int32_t j = cok ? c - sl * gc.ncols : 0;
            const int32_t s = s0 + sl;
            const int64_t t_out0 = steps_of(a.batch, s) * op.out_u;
            // fused unit, first result: act2(scale1 * acc + bias1) rounded into
            // this column's row of the 1x1 conv's A operand (rows of 128
            // channels in two 64-channel K slices, 128-byte swizzled)
            bool waited = !bar_red_or(*abort_flag != 0) && mbar_wait(tfull + buf, (tile_j >> 1) & 1, a.wait_ns);
            waited = !bar_red_or(!waited);
            if (!waited) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + buf * 256;
            if (op.k2 > 0) {
              const int32_t nh = op.N / 2;  // rows per half (the first conv's channels)
              for (int32_t n0 = half * nh; n0 < (half + 1) * nh; n0 += 16) {
                uint32_t v[16];
                tmem_ld16(lane_base + n0, v);
                tmem_ld_wait();
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  float y0 = fmaf(__uint_as_float(v[2 * q]), __ldg(op.scale + n0 + 2 * q), op.bias ? __ldg(op.bias + n0 + 2 * q) : 0.f);
                  float y1 = fmaf(__uint_as_float(v[2 * q + 1]), __ldg(op.scale + n0 + 2 * q + 1),
                                  op.bias ? __ldg(op.bias + n0 + 2 * q + 1) : 0.f);
                  if (op.act2) {
                    y0 = leaky(y0);
                    y1 = leaky(y1);
                  }
                  pk[q] = pack_lp(y0, y1, lp_bf16);
                }
                // channels n0 .. n0+15: K slice n0 / 64, 16-byte chunks (n0 % 64) / 8 and +1
                uint8_t* row = sU + (n0 >> 6) * kTile + r * 128;
                const int chunk = (n0 & 63) >> 3;
                *reinterpret_cast<uint4*>(row + (((chunk) ^ (r & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(row + (((chunk + 1) ^ (r & 7)) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
              }
              fence_proxy_async_smem();
              epi_sync();
              if (t == 0) mbar_arrive(b2ready);
              bool w2 = mbar_wait(tfull2 + buf, fused_use[buf] & 1, a.wait_ns);
              ++fused_use[buf];
              w2 = !bar_red_or(!w2);
              if (!w2) {
                ok = false;
                break;
              }
              tc_fence_after();
            }
            // the stored result: acc (second accumulator for a fused unit) x
            // scale + bias (+ the aligned residual), every view
            const uint32_t acc = lane_base + (op.k2 > 0 ? 128 : 0);
            const float* sc = op.k2 > 0 ? op.scale2 : op.scale;
            const float* bi = op.k2 > 0 ? op.bias2 : op.bias;
            const int32_t nrows = op.k2 > 0 ? op.N2 : op.N;  // MMA N (rows rounded up to 16)
            const int32_t mrows = op.k2 > 0 ? op.M2 : op.M;  // real rows
            const int32_t nh = nrows / 2;
            char* base = slot_base(a.batch, s);
            for (int32_t n0 = half * nh; n0 < (half + 1) * nh; n0 += 8) {
              uint32_t v[8];
              tmem_ld8(acc + n0, v);
              tmem_ld_wait();
              if (!cok || n0 >= mrows) continue;
              const int32_t ph = op.phases > 1 ? n0 / op.cout : 0;
              const int32_t ch = n0 - ph * op.cout;
              const int64_t tb = t_out0 + (int64_t)j * op.phases + ph;
              float x[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) x[q] = fmaf(__uint_as_float(v[q]), __ldg(sc + n0 + q), bi ? __ldg(bi + ch + q) : 0.f);
              if (op.has_skip) {
                const float* sk = reinterpret_cast<const float*>(base + op.skip.off) +
                                  ring_row(tb - op.skip_A, op.skip.rows) * op.skip.chans + op.skip.choff + ch;
                const float4 a0 = *reinterpret_cast<const float4*>(sk);
                const float4 a1 = *reinterpret_cast<const float4*>(sk + 4);
                x[0] += a0.x; x[1] += a0.y; x[2] += a0.z; x[3] += a0.w;
                x[4] += a1.x; x[5] += a1.y; x[6] += a1.z; x[7] += a1.w;
              }
              if (op.is_last) {
                float* e = a.ext + (int64_t)s * a.ext_stride + ((int64_t)j * op.phases + ph) * op.cout + ch;
#pragma unroll
                for (int q = 0; q < 8; ++q) e[q] = x[q];
              }
              const Ring& f = op.out.f32;
              if (f.rows) {
                float* pf = reinterpret_cast<float*>(base + f.off) + ring_row(tb, f.rows) * f.chans + f.choff + ch;
                st_global_v4(pf, make_uint4(__float_as_uint(x[0]), __float_as_uint(x[1]), __float_as_uint(x[2]),
                                            __float_as_uint(x[3])));
                st_global_v4(pf + 4, make_uint4(__float_as_uint(x[4]), __float_as_uint(x[5]), __float_as_uint(x[6]),
                                                __float_as_uint(x[7])));
              }
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const Ring& lr = op.out.lp[q];
                if (!lr.rows) continue;
                float y[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) y[e] = q ? leaky(x[e]) : x[e];
                const uint4 pk = make_uint4(pack_lp(y[0], y[1], lp_bf16), pack_lp(y[2], y[3], lp_bf16),
                                            pack_lp(y[4], y[5], lp_bf16), pack_lp(y[6], y[7], lp_bf16));
                const int64_t row = ring_row(tb, lr.rows);
                char* pl = base + lr.off + (row * lr.chans + ch) * 2;
                st_global_v4(pl, pk);
                if (row >= lr.rows - lr.pre) st_global_v4(pl - (int64_t)lr.rows * lr.chans * 2, pk);  // mirror
              }
            }
            // the accumulator buffer is free for the tile after next
            tc_fence_before();
            epi_sync();
            if (t == 0) mbar_arrive(tempty + buf);
          }
          if (!ok) break;
        } else if (op.kind == kTailConv32) {
          // narrow FP32 convolution / polyphase transposed convolution: one
          // (column, row) item per thread at a time, reduction over (tap, channel)
          const int64_t items = (int64_t)ncol_g * op.M;
          for (int64_t it = t; it < items; it += kTailEpi) {
            const int32_t c = (int32_t)(it / op.M), m = (int32_t)(it - (int64_t)c * op.M);
            const int32_t sl = c / gc.ncols, j = c - sl * gc.ncols, s = s0 + sl;
            const char* base = slot_base(a.batch, s);
            const float* in = reinterpret_cast<const float*>(base + op.in.off) + op.in.choff;
            const int64_t t0 = steps_of(a.batch, s) * op.in.u + j - op.hist;
            const float* w = op.A32 + (int64_t)m * op.Kt;
            float acc = 0.f;
            for (int32_t tap = 0; tap < op.taps; ++tap) {
              const float* xr = in + ring_row(t0 + (int64_t)tap * op.dil, op.in.rows) * op.in.chans;
              for (int32_t ci = 0; ci < op.cin; ++ci) acc = fmaf(__ldg(w + tap * op.cin + ci), activate(xr[ci], op.act), acc);
            }
            const int32_t ph = op.phases > 1 ? m / op.cout : 0;
            const int32_t ch = m - ph * op.cout;
            const int64_t tb = steps_of(a.batch, s) * op.out_u + (int64_t)j * op.phases + ph;
            float v = acc + (op.bias ? __ldg(op.bias + ch) : 0.f);
            if (op.has_skip)
              v += reinterpret_cast<const float*>(base + op.skip.off)[ring_row(tb - op.skip_A, op.skip.rows) *
                                                                          op.skip.chans + op.skip.choff + ch];
            put_value(op, a, s, tb, (int64_t)j * op.phases + ph, ch, v);
          }
        } else if (op.kind == kTailHeads) {
          const int64_t items = (int64_t)ncol_g * op.bands;
          for (int64_t it = t; it < items; it += kTailEpi) {
            const int32_t c = (int32_t)(it / op.bands), b = (int32_t)(it - (int64_t)c * op.bands);
            const int32_t sl = c / gc.ncols, j = c - sl * gc.ncols, s = s0 + sl;
            const char* base = slot_base(a.batch, s);
            const int64_t tb = steps_of(a.batch, s) * op.out_u + j;
            float v[3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
              v[q] = reinterpret_cast<const float*>(base + op.hin[q].off)[ring_row(tb - op.hA[q], op.hin[q].rows) *
                                                                               op.hin[q].chans + op.hin[q].choff + b];
            float y = tanhf(v[0]) * sigmoid_f(v[1]);
            if (op.noise)
              y += sigmoid_f(v[2]) * noise_uniform(a.batch.seeds[a.batch.slots[s]], tb - op.hdelay, b, op.bands);
            put_value(op, a, s, tb, j, b, y);
          }
        } else if (op.kind == kTailAdd) {
          const int64_t items = (int64_t)ncol_g * op.cout;
          for (int64_t it = t; it < items; it += kTailEpi) {
            const int32_t c = (int32_t)(it / op.cout), ch = (int32_t)(it - (int64_t)c * op.cout);
            const int32_t sl = c / gc.ncols, j = c - sl * gc.ncols, s = s0 + sl;
            const char* base = slot_base(a.batch, s);
            const int64_t tb = steps_of(a.batch, s) * op.out_u + j;
            float y = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q)
              y += reinterpret_cast<const float*>(base + op.hin[q].off)[ring_row(tb - op.hA[q], op.hin[q].rows) *
                                                                             op.hin[q].chans + op.hin[q].choff + ch];
            put_value(op, a, s, tb, j, ch, y);
          }
        }
        // op complete for this group: its stores visible to the next op's
        // window loads (async proxy) and plain loads
        fence_proxy_async_global();
        epi_sync();
        ++op_count;
        if (t == 0) st_release_smem(ops_completed, op_count);
      }
      if (!ok) break;
      // the group's streams advance by this call's steps (every op of the group
      // has read its step counter)
      epi_sync();
      if (a.advance && t < gs) const_cast<int64_t*>(a.batch.counters)[a.batch.slots[s0 + t]] += a.steps;
    }
    if (!ok) {
      *abort_flag = 1;
      if (t == 0) atomicOr(a.err, 2);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

}  // namespace

cudaError_t launch_tail(const TailArgs& a, int grid, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (a.batch.count <= 0) return cudaSuccess;
  return launch_pdl(k_tail, dim3((unsigned)grid), dim3(kTailThreads), (size_t)kTailSmem, st, a);
}

}  // namespace cc
