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
//              window rows in the 128-byte-swizzled operand layout.  When the
//              tile's streams occupy consecutive slots at the same step, the
//              rows of 128 columns are one 3D box (frames x slots) of the
//              input view; otherwise they are gathered four at a time
//              (tile::gather4), which costs about four times as much per
//              slice.  One expect-tx per stage, no thread waits on its own
//              copies, so every stage can be in flight
//   warp 1     TMEM allocation; lane 0 issues tcgen05.mma (128 x BN x 16,
//              BF16 or FP16 operands, FP32 accumulation in TMEM)
//   warps 2..  epilogue (EW = 8 or 16 warps): warp w owns accumulator rows
//              32*(w%4) .. +31 (its TMEM lane quarter) and every (EW/4)-th
//              group of 8 columns (the warps of a quarter interleave); per
//              group it loads the rows (tcgen05.ld), applies scale and bias,
//              turns the 32 x 8 block around in 1 KB of shared memory so that
//              each lane holds 8 consecutive channels of one column, adds the
//              aligned residual (16-byte loads) and stores every view with
//              16-byte stores, at ring addresses from a per-column table built
//              before the kernel waits on its predecessor.  A layer of at most
//              64 rows stores its weight tiles twice (rows 64..127 repeat
//              0..63), so lane quarters 2 and 3 hold the same results and
//              their warps store every other 32-column chunk: no epilogue
//              warp idles on the padding rows
// Residual-unit fusion (FUSE): a k-wide conv and the 1x1 conv that consumes
// only it run as one launch.  The first epilogue writes the scaled, biased,
// activated first result in BF16/FP16 straight into shared memory in the
// swizzled K-major operand layout; the MMA warp then runs the 1x1 contraction
// (its weights streamed through the same pipeline) into a second TMEM
// accumulator, and the second epilogue is the ordinary one.  The rounding of
// the intermediate is the one the unfused path applies when it stores it, so
// the results are identical.  The unit's residual (its input, written by the
// previous launch) is copied (cp.async) into the B stages as soon as the first
// contraction has drained them, so the second epilogue reads it from shared
// memory instead of waiting on L2 once per 8-column group.
// Split-K (layers with few tiles and long K): the ksplit CTAs of a cluster
// along z share one tile; CTA z accumulates an equal share of the K slices and
// finishes columns [z, z+1) * BN/ksplit.  Each CTA pushes its partial sums of
// the other CTAs' columns into their shared memory (distributed shared-memory
// stores); after one cluster barrier, each CTA adds its own partial (TMEM) and
// the received ones in the fixed order z = 0, 1, ...  The split is a property
// of the layer, so a stream's result does not depend on the batch it runs in.
// Every mbarrier wait is bounded in time and records an error in the model's
// device error word instead of hanging.
//
// Reads before griddepcontrol.wait: the weights, scales and biases (written at
// model creation), the batch's slot list and step counters, and (skip_early)
// the residual rows.  Every kernel of a launch chain issues
// griddepcontrol.launch_dependents only after its own wait, so when a grid
// starts, every launch before its predecessor has completed: the slot list
// (uploaded before the chain), the counters (advanced by the previous chain's
// last kernel) and a residual produced two or more launches back are final.
#include <cuda.h>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_sm100.cuh"

namespace cc {
namespace {

using namespace sm100;

constexpr int kBM = 128;

// Variants (launch_conv_tc): threads = producer warp + MMA warp + EW epilogue
// warps.  128-column tiles run 6 stages and 16 epilogue warps (one CTA per SM:
// few CTAs with long K loops need deep prefetch, and the epilogue has the SM
// to itself) when the grid fits in one wave and the model expects no
// concurrent launch chains; else 3 stages and 8 epilogue warps (two CTAs per
// SM, whose epilogues overlap each other's main loops and other chains'
// kernels).  Split layers run 4 stages with a receive buffer; fused units 4
// or 2 stages with the second operand; 256-column tiles 4 stages.
template <int BN, int STAGES, bool FUSE, int EW, bool SPLIT = false, int MT = 1>
struct TcLayout {
  static constexpr int kThreads = 64 + 32 * EW;
  static constexpr int kStages = STAGES;
  static constexpr int kA = kBM * 128;  // one 128 x 64 low-precision tile
  static constexpr int kB = BN * 128;
  static constexpr int kBars = (2 * kStages + 1) * 8 + 8;
  // column table per view (f32, lp0, lp1, skip): arena offset in 16-byte
  // units of the ring row holding the column's first frame, that ring row,
  // the mirror row's offset (low-precision views); the caller-buffer offset
  static constexpr int kCols = BN * (4 * 4 + 4 * 4 + 2 * 4 + 8);
  static constexpr int kTurn = EW * 32 * 8 * 4;  // per epilogue warp: 32 rows x 8 columns of FP32
  // fused unit: the 1x1 conv's operand, BN columns x 128 * MT channels (2 * MT
  // K slices; MT > 1: the unit's channels span MT M tiles of a cluster)
  static constexpr int kB2 = FUSE ? 2 * MT * BN * 128 : 0;
  static constexpr int kBars2 = FUSE ? 16 : 0;          // b2ready, tfull2
  // split-K receive buffer: the other CTAs' partials of this CTA's columns
  // ([ksplit-1][BN/ksplit][128] FP32: at most 3 x 32 or 1 x 64 columns)
  static constexpr int kRecv = SPLIT ? 3 * (BN / 4) * kBM * 4 : 0;
  static constexpr int kBytes = 1024 + kStages * (kA + kB) + kB2 + kRecv + kBars + kBars2 + kCols + kTurn + 64;
  static constexpr int kMinBlocks = (STAGES == 3 || (FUSE && STAGES == 2)) ? 2 : 1;
  static constexpr int kTmemCols = FUSE ? 2 * BN : BN;
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi, bool bf16) {
  if (bf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int BN, int STAGES, bool FUSE, int EW, bool SPLIT, int MT>
__global__ void __launch_bounds__(TcLayout<BN, STAGES, FUSE, EW, SPLIT, MT>::kThreads,
                                  TcLayout<BN, STAGES, FUSE, EW, SPLIT, MT>::kMinBlocks)
    k_conv_tc(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmB,
              const TcArgs a) {
  using L = TcLayout<BN, STAGES, FUSE, EW, SPLIT, MT>;
  constexpr int kEpi = 32 * EW;  // epilogue threads
  constexpr int kParts = EW / 4;  // epilogue warps per TMEM lane quarter
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * L::kA;
  uint8_t* sB2 = sB + kStages * L::kB;  // fused unit: second operand (1024-aligned)
  float* const recv = reinterpret_cast<float*>(sB2 + L::kB2);  // split-K receive buffer
  uint64_t* full = reinterpret_cast<uint64_t*>(sB2 + L::kB2 + L::kRecv);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* b2ready = tfull + 1;  // fused unit (FUSE only)
  uint64_t* tfull2 = tfull + 2;
  uint32_t* tbase = reinterpret_cast<uint32_t*>(tfull + 1 + (FUSE ? 2 : 0));
  int64_t* col_ext = reinterpret_cast<int64_t*>(tbase + 2);   // [BN]
  uint32_t* col_off = reinterpret_cast<uint32_t*>(col_ext + BN);  // [4][BN], 16-byte units
  int32_t* col_row = reinterpret_cast<int32_t*>(col_off + 4 * BN);  // [4][BN]
  uint32_t* col_mir = reinterpret_cast<uint32_t*>(col_row + 4 * BN);  // [2][BN], ~0u: none
  float* turn = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(col_mir + 2 * BN) + 15) & ~static_cast<uintptr_t>(15));  // [8 warps][8][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t m0 = blockIdx.y * kBM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  const int nk = a.Kt / 64;
  const int cchunks = a.cin / 64;
  const int KS = SPLIT ? (int)gridDim.z : 1, zr = SPLIT ? (int)blockIdx.z : 0;  // split-K (cluster along z)
  const int kb = zr * nk / KS, ke = (zr + 1) * nk / KS;  // this CTA's K slices
  const int c_n = BN / KS, c_lo = zr * c_n;              // columns this CTA finishes

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);  // the producer's expect-tx arrival; TMA completes the bytes
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull, 1);
    if (FUSE) {
      mbar_init(b2ready, 1);
      mbar_init(tfull2, 1);
    }
    fence_mbar_init();
    prefetch_tmap(a.box_ok ? &tmT : &tmB);
  }
  // Producer set-up before the CTA barrier: the batch's slots and step
  // counters are loaded while thread 0 initialises the barriers and warp 1
  // allocates TMEM.  For most CTAs of a one-wave launch this runs when the
  // previous launch's CTA on the SM exits, on the chain's critical path.
  const int nks = ke - kb;
  const int pre = nks < kStages ? nks : kStages;
  const uint8_t* atile = static_cast<const uint8_t*>(a.A_tiled) + ((size_t)blockIdx.y * nk + kb) * L::kA;
  constexpr int G = BN / 128;
  bool boxes = false;
  int32_t by[G], bz[G];
  if (warp == 0) {
    // Box form: the streams of the tile sit in consecutive slots at one step p,
    // and the call's frames do not cross the ring's end; then tap k's rows of
    // the 128 columns of half g start at view row pre + p - hist + j_g + k*dil
    // of slot bz[g] (the mirrored tail holds the rows before ring row 0).
    if (a.box_ok) {
      const int64_t s_first = n0 / a.ncols;
      const int64_t s_end = min((n0 + BN - 1) / a.ncols + 1, (int64_t)a.batch.count);
      // A tile spans at most BN streams; lane l checks streams s_first + l +
      // 32 i.  Every slot is loaded at once, then every step counter: two
      // dependent round trips to L2.
      constexpr int kIt = BN / 32;
      int32_t sl[kIt];
      int64_t sp[kIt];
#pragma unroll
      for (int i = 0; i < kIt; ++i) {
        const int64_t s = s_first + lane + 32 * i;
        sl[i] = s < s_end ? a.batch.slots[s] : 0;
      }
#pragma unroll
      for (int i = 0; i < kIt; ++i) {
        const int64_t s = s_first + lane + 32 * i;
        sp[i] = s < s_end ? a.batch.counters[sl[i]] : 0;
      }
      const int32_t slot0 = __shfl_sync(0xffffffffu, sl[0], 0);  // stream s_first (lane 0, i = 0)
      const int64_t step0 = shfl64(sp[0], 0);
      bool reg = true;
#pragma unroll
      for (int i = 0; i < kIt; ++i) {
        const int64_t s = s_first + lane + 32 * i;
        if (s < s_end) reg = reg && sl[i] == slot0 + (int32_t)(s - s_first) && sp[i] == step0;
      }
      const int32_t p = (int32_t)ring_row(step0 * a.in.u, a.in.rows);
      boxes = __all_sync(0xffffffffu, reg) && p + a.ncols <= a.in.rows;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int64_t ng = n0 + 128 * g;
        const int64_t sg = ng / a.ncols;
        by[g] = a.in.pre + p - a.hist + (int32_t)(ng - sg * a.ncols);
        bz[g] = slot0 + (int32_t)(sg - s_first);
      }
    }
  }
  if (warp == 1) {
    tmem_alloc(tbase, L::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  // a cluster-fused unit writes into its peers' shared memory: every thread
  // arrives here, and each waits on this phase (every CTA of the cluster has
  // started) before its part in the operand exchange
  if (FUSE && MT > 1) cluster_arrive();

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // the weight tiles of the first stages
    if (lane == 0)
      for (int i = 0; i < pre; ++i) {
        mbar_arrive_expect_tx(full + i, L::kA + L::kB);
        bulk_load(sA + i * L::kA, atile + (size_t)i * L::kA, L::kA, full + i);
      }
    // gather form: lane l gathers tile rows 4*(l + 32*g) .. +3 for g < G
    int32_t ybase[G][4], r0[G][4];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t n = n0 + 4 * (lane + 32 * g) + i;
        ybase[g][i] = 0;
        r0[g][i] = -1;  // column past the batch: read arena row 0, result discarded
        if (!boxes && n < N) {
          const int32_t s = (int32_t)(n / a.ncols);
          const int32_t j = (int32_t)(n - (int64_t)s * a.ncols);
          ybase[g][i] = a.batch.slots[s] * a.in_rows_per_slot + a.in_row_off;
          r0[g][i] = (int32_t)ring_row(steps_of(a.batch, s) * a.in.u + (int64_t)j * a.stride - a.hist,
                                       a.in.rows);
        }
      }
    pdl_wait();  // the input view is the previous launch's output
    pdl_release();
    // failure-detection test hook: while the model's withhold counter is
    // positive, the first CTA of a launch takes one off it and leaves the
    // window rows of its first K slice unrequested, so its pipeline waits run
    // out after wait_ns (no copy is left in flight: the slice's weight tile
    // lands, its expected bytes never complete)
    bool withhold = false;
    if (a.withhold && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
      int take = 0;
      if (lane == 0 && *reinterpret_cast<volatile int32_t*>(a.withhold) > 0) take = atomicSub(a.withhold, 1) > 0;
      withhold = __shfl_sync(0xffffffffu, take, 0) != 0;
    }
    bool ok = true;
    int issued = 0;
    for (int i = 0; i < nks; ++i) {
      const int kc = kb + i;
      const int st = i % kStages;
      const uint32_t ph = (i / kStages) & 1;
      if (!mbar_wait(empty + st, ph ^ 1, a.wait_ns)) {
        ok = false;
        break;
      }
      const int tap = kc / cchunks;
      const int c0 = (kc - tap * cchunks) * 64;
      if (lane == 0 && i >= pre) {
        mbar_arrive_expect_tx(full + st, L::kA + L::kB);
        bulk_load(sA + st * L::kA, atile + (size_t)i * L::kA, L::kA, full + st);
      }
      __syncwarp();
      uint8_t* dst = sB + st * L::kB;
      if (i == 0 && withhold) {
        // failure-detection test: this slice's rows are never requested
      } else if (boxes) {
        if (lane == 0)
#pragma unroll
          for (int g = 0; g < G; ++g) tma_load_3d(dst + g * 16384, &tmT, full + st, c0, by[g] + tap * a.dil, bz[g]);
      } else {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          int32_t y[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            y[i] = r0[g][i] < 0 ? 0 : ybase[g][i] + wrap_row(r0[g][i] + tap * a.dil, a.in.rows);
          tma_gather4(dst + (lane + 32 * g) * 512, &tmB, full + st, c0, y[0], y[1], y[2], y[3]);
        }
      }
      issued = i + 1;
    }
    if (FUSE && ok) {
      // fused unit: the 1x1 conv's weight slices through the same stages
      const uint8_t* a2tile = static_cast<const uint8_t*>(a.A2_tiled) + (size_t)blockIdx.y * a.k2 * L::kA;
      for (int j = 0; j < a.k2; ++j) {
        const int i = nks + j;
        const int st = i % kStages;
        const uint32_t ph = (i / kStages) & 1;
        if (!mbar_wait(empty + st, ph ^ 1, a.wait_ns)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_arrive_expect_tx(full + st, L::kA);
          bulk_load(sA + st * L::kA, a2tile + (size_t)j * L::kA, L::kA, full + st);
        }
        __syncwarp();
        issued = i + 1;
      }
    }
    // every copy this warp issued lands before the CTA's shared memory goes
    // away: normally the MMA warp has already seen them complete; after a
    // wait that gave up (here or in the MMA warp) the stages still in flight
    // are waited for, again within the limit
    bool drained = true;
    for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
      drained = mbar_wait(full + i % kStages, (i / kStages) & 1, a.wait_ns) && drained;
    if ((!ok || !drained) && lane == 0) atomicOr(a.err, 1);
    if (KS > 1) cluster_sync();  // the epilogue's partial exchange
    if (FUSE && MT > 1) {
      // the first epilogue's operand exchange: this warp takes no part but
      // must arrive (every thread of the cluster does)
      cluster_wait();
      cluster_arrive();
      cluster_wait();
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    pdl_wait();
    pdl_release();
    const uint32_t idesc = idesc_f16(kBM, BN, a.in.dtype == kDtBF16);
    bool ok = true;
    if (lane == 0) {
      for (int i = 0; i < ke - kb; ++i) {
        const int st = i % kStages;
        const uint32_t ph = (i / kStages) & 1;
        if (!mbar_wait(full + st, ph, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(sA + st * L::kA), sb = smem_u32(sB + st * L::kB);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_f16(tmem, sw128_kmajor_desc(sa + k * 32), sw128_kmajor_desc(sb + k * 32), idesc,
                  (i | k) != 0);
        mma_commit(empty + st);
      }
      mma_commit(tfull);
    }
    __syncwarp();
    // the operand exchange of a cluster-fused unit: arrive before waiting for
    // the operand (the epilogues' barrier needs every thread of the cluster)
    if (FUSE && MT > 1) {
      cluster_wait();
      cluster_arrive();
    }
    if (FUSE && lane == 0) {
      // fused unit: wait for the first epilogue's operand, then the 1x1 conv
      // into the second accumulator (TMEM columns BN .. 2*BN-1)
      ok = ok && mbar_wait(b2ready, 0, a.wait_ns);
      tc_fence_after();
      const int nks = ke - kb;
      for (int j = 0; ok && j < a.k2; ++j) {
        const int i = nks + j;
        const int st = i % kStages;
        const uint32_t ph = (i / kStages) & 1;
        if (!mbar_wait(full + st, ph, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(sA + st * L::kA), sb = smem_u32(sB2 + j * BN * 128);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_f16(tmem + BN, sw128_kmajor_desc(sa + k * 32), sw128_kmajor_desc(sb + k * 32), idesc,
                  (j | k) != 0);
        mma_commit(empty + st);
      }
      mma_commit(tfull2);
    }
    if (lane == 0 && !ok) atomicOr(a.err, 4);
    __syncwarp();
    if (FUSE && MT > 1) cluster_wait();
    if (KS > 1) cluster_sync();  // the epilogue's partial exchange
  } else {
    // ---------------------------------------------------------------- epilogue
    const int t = threadIdx.x - 64;  // 0..255
    const int sub = warp & 3;        // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // which groups of 8 columns: half, half + kParts, ...
    // Repeated rows (TcArgs::mdup; not with split-K or cluster tiles): lane
    // quarters 2 and 3 hold rows 0..63 again, and the two quarter pairs take
    // alternate 32-column chunks (alternate kParts-group runs in the fused
    // unit's first epilogue)
    const bool dup = !SPLIT && MT == 1 && a.mdup != 0;
    const int rsub = dup ? (sub & 1) : sub;  // rows 32*rsub .. +31 of the tile
    const int rpart = dup ? (sub >> 1) : 0;
    const int nrep = dup ? 2 : 1;
    const int32_t m = m0 + rsub * 32 + lane;  // accumulator row of this thread
    const bool mok = m < a.M;
    const int32_t ph = (mok && a.phases > 1) ? m / a.cout : 0;  // transposed conv: phase
    const int32_t ch = mok ? m - ph * a.cout : 0;                // output channel
    const float sc1 = mok ? a.scale[m] : 0.f;
    const float bi1 = (mok && a.bias) ? a.bias[ch] : 0.f;
    // the stored result's scale and bias (the fused unit's second conv)
    const float sc = !FUSE ? sc1 : mok ? a.scale2[m] : 0.f;
    const float bi = !FUSE ? bi1 : (mok && a.bias2) ? a.bias2[ch] : 0.f;
    // Column table (pre-wait): per view, the 16-byte-unit arena offset of the
    // ring row holding the column's first frame and that row; for a
    // low-precision view also the offset of its mirror row (~0u if the row is
    // not in the mirrored tail; used when phases == 1).  The arena is below
    // 64 GiB, so offsets fit 32 bits.
    for (int c = t; c < BN; c += kEpi) {
      const int64_t n = n0 + c;
      if (n >= N) break;
      const int32_t s = (int32_t)(n / a.ncols);
      const int32_t j = (int32_t)(n - (int64_t)s * a.ncols);
      const int64_t sb = (int64_t)a.batch.slots[s] * a.batch.slot_bytes;
      const int64_t tb = steps_of(a.batch, s) * a.out_u + (int64_t)j * a.phases;
      col_ext[c] = (int64_t)s * a.out.ext_stride + (int64_t)j * a.phases * a.cout;
      auto put = [&](int v, int64_t off, int32_t rows, int32_t chans, int32_t pre, int64_t time, int elem) {
        const int32_t row = rows ? (int32_t)ring_row(time, rows) : 0;
        const int64_t pitch = (int64_t)chans * elem;
        col_row[v * BN + c] = row;
        col_off[v * BN + c] = (uint32_t)((sb + off + row * pitch) >> 4);
        if (v == 1 || v == 2)
          col_mir[(v - 1) * BN + c] = (rows && row >= rows - pre) ? (uint32_t)((sb + off + (row - rows) * pitch) >> 4) : ~0u;
      };
      put(0, a.out.f32.off, a.out.f32.rows, a.out.f32.chans, 0, tb, 4);
      put(1, a.out.lp[0].off, a.out.lp[0].rows, a.out.lp[0].chans, a.out.lp[0].pre, tb, 2);
      put(2, a.out.lp[1].off, a.out.lp[1].rows, a.out.lp[1].chans, a.out.lp[1].pre, tb, 2);
      put(3, a.skip.off + (int64_t)a.skip.choff * 4, a.skip.rows, a.skip.chans, 0, tb - a.skip_A, 4);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");  // column table complete
    char* const arena = a.batch.arena;
    const bool phased = a.phases > 1;
    // After the turn, lane l holds column kk = l / 4 of its group and the 8
    // consecutive rows 8*(l % 4) .. +7 of its warp's 32: channels ch_l .. +7
    // of phase ph_l (cout is a multiple of 8, so they share a phase).
    const int kk = lane >> 2;
    const int32_t mrow = m0 + rsub * 32 + 8 * (lane & 3);
    const bool vok = mrow < a.M;
    const int32_t ph_l = (vok && phased) ? mrow / a.cout : 0;
    const int32_t ch_l = vok ? mrow - ph_l * a.cout : 0;
    float* const tw = turn + (warp - 2) * 256;
    // Offset (16-byte units) of this lane's row of a column for a phased
    // (transposed) layer: the column's first row + ph_l, wrapped at the ring end.
    auto phase_off = [&](uint32_t o16, int32_t row, int32_t rows, int32_t pitch16) -> uint32_t {
      return o16 + (uint32_t)((row + ph_l >= rows ? ph_l - rows : ph_l) * pitch16);
    };
    const int32_t s_rows = a.skip.rows, s_p16 = a.skip.chans / 4;
    char* const sk_base = arena + (int64_t)ch_l * 4;
    // residual rows of the tile: every 128-byte line into L2 ahead of use
    auto prefetch_skip = [&]() {
      for (int c = c_lo + t; c < c_lo + c_n; c += kEpi) {
        if (n0 + c >= N) break;
        for (int k = 0; k < kBM; k += 32) {
          const int32_t mm = m0 + k;
          if (mm >= a.M) break;
          const int32_t p2 = a.phases > 1 ? mm / a.cout : 0;
          const int32_t row = col_row[3 * BN + c];
          const int32_t d = row + p2 >= s_rows ? p2 - s_rows : p2;
          prefetch_l2(arena + (uint64_t)col_off[3 * BN + c] * 16 + ((int64_t)d * a.skip.chans + (mm - p2 * a.cout)) * 4);
        }
      }
    };
    // Columns go in groups of 8 inside chunks of 32: per chunk lane l holds
    // the table entries of column cb + l; a group's lanes fetch those of their
    // column by one shuffle per view.  Residual values of the next group are
    // requested before the current group's stores.
    float4 sk0 = make_float4(0.f, 0.f, 0.f, 0.f), sk1 = sk0;
    auto load_skip = [&](int cb, int g, uint32_t so, int32_t sr) {
      uint32_t o = __shfl_sync(0xffffffffu, so, 8 * g + kk);
      const int32_t rw = __shfl_sync(0xffffffffu, sr, 8 * g + kk);
      if (phased) o = phase_off(o, rw, s_rows, s_p16);
      const bool ok = vok && n0 + cb + 8 * g + kk < N;
      const char* pa = sk_base + (uint64_t)o * 16;
      sk0 = ok ? ld_global_nc_v4(pa) : make_float4(0.f, 0.f, 0.f, 0.f);
      sk1 = ok ? ld_global_nc_v4(pa + 16) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // Fused unit: the residual tile (this tile's rows, FP32, a column per
    // stg_rows * 4 bytes, 16-byte chunks XOR-swizzled by the column's parity)
    // is copied into the B stages, free once the first contraction is done,
    // while the first epilogue and the 1x1 MMAs run
    const int stg_rows = a.M - m0 <= 64 ? 64 : 128;
    const bool staged = FUSE && a.has_skip && BN * stg_rows * 4 <= kStages * L::kB;
    const int cstep = 32 * nrep;  // chunk stride of this warp's column chunks
    uint32_t so_next = 0;
    int32_t sr_next = 0;
    if (a.has_skip) {
      so_next = col_off[3 * BN + c_lo + 32 * rpart + lane];
      sr_next = col_row[3 * BN + c_lo + 32 * rpart + lane];
    }
    if (a.has_skip && a.skip_early) {
      prefetch_skip();
      if (!staged) load_skip(c_lo + 32 * rpart, half, so_next, sr_next);
    }
    pdl_wait();
    pdl_release();
    if (a.has_skip && !a.skip_early) {
      prefetch_skip();
      if (!staged) load_skip(c_lo + 32 * rpart, half, so_next, sr_next);
    }
    // one outcome for all epilogue threads (a reduction barrier), so the
    // named barriers stay matched
    const bool waited = mbar_wait(tfull, 0, a.wait_ns);
    uint32_t all_ok;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(all_ok)
        : "r"((uint32_t)waited), "n"(kEpi)
        : "memory");
    tc_fence_after();
    if (staged && all_ok) {
      // every MMA that read the B stages has completed (tfull)
      const int nq = stg_rows / 4;
      const uint32_t sdst = smem_u32(sB);
      for (int i = t; i < BN * nq; i += kEpi) {
        const int c = i / nq, q = i - c * nq;
        if (n0 + c >= N) break;
        if (m0 + 4 * q >= a.M) continue;
        cp_async16(sdst + (uint32_t)(c * stg_rows * 4 + ((q ^ (c & 1)) << 4)),
                   arena + (uint64_t)col_off[3 * BN + c] * 16 + (int64_t)(m0 + 4 * q) * 4);
      }
      cp_async_commit();
    }
    uint32_t acc_col = 0;  // TMEM column of the stored result's accumulator
    if (FUSE) {
      // fused unit, first epilogue: the k-wide conv's result, scaled, biased,
      // activated and rounded, into the 1x1 conv's K-major operand (row =
      // column of the tile, 128-byte-swizzled rows, 64 channels per K slice)
      // Each lane holds one channel (its accumulator row) of 8 columns: it
      // stores 2 bytes per column; a warp's 32 channels of a column are four
      // 16-byte chunks of that column's swizzled row.
      const bool lp_bf16 = a.in.dtype == kDtBF16;
      const int32_t cm = m;  // channel = accumulator row (phases == 1)
      uint8_t* const b2row = sB2 + (cm >> 6) * (BN * 128) + (cm & 7) * 2;
      const int chunk1 = (cm & 63) >> 3;
      if (MT > 1) cluster_wait();  // every peer has started
      if (all_ok)
#pragma unroll 1
        for (int g = half + kParts * rpart; g < BN / 8; g += kParts * nrep) {
          uint32_t r[8];
          tmem_ld8(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(8 * g), r);
          tmem_ld_wait();
          if (mok)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              float y = fmaf(__uint_as_float(r[k]), sc1, bi1);
              if (a.act2) y = leaky(y);
              const uint16_t h = lp_bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(y))
                                         : __half_as_ushort(__float2half_rn(y));
              const int c = 8 * g + k;
              uint8_t* const dst = b2row + c * 128 + ((chunk1 ^ (c & 7)) << 4);
              if (MT == 1) {
                *reinterpret_cast<uint16_t*>(dst) = h;
              } else {
                // every CTA of the cluster multiplies the whole intermediate
                const uint32_t sa = smem_u32(dst);
#pragma unroll
                for (int q = 0; q < MT; ++q) dsmem_st_u16(dsmem_map(sa, (uint32_t)q), h);
              }
            }
        }
      // the operand is read by the tensor cores (async proxy)
      if (MT > 1)
        fence_proxy_async_cluster();
      else
        fence_proxy_async_smem();
      if (MT > 1) {
        // every CTA's channels are in every CTA's operand after this
        cluster_arrive();
        cluster_wait();
        fence_proxy_async_smem();
      } else {
        asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");
      }
      if (t == 0) mbar_arrive(b2ready);
      // the staged residual: own copies complete here, everyone's after the
      // barrier below
      if (staged) cp_async_wait_all();
      const bool waited2 = mbar_wait(tfull2, 0, a.wait_ns);
      uint32_t ok2;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\t"
          "setp.ne.u32 q, %1, 0;\n\t"
          "bar.red.and.pred p, 1, %2, q;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok2)
          : "r"((uint32_t)waited2), "n"(kEpi)
          : "memory");
      tc_fence_after();
      all_ok = all_ok && ok2;
      acc_col = BN;
    }
    // split-K: receive buffer [KS-1 senders][c_n columns][128 rows] FP32 of
    // its own (never touched by the main loop, so a CTA may push into a
    // slower one's); sender z's slot in owner o's buffer is z (z < o) or z - 1
    if (SPLIT && KS > 1) {
      if (all_ok)
        for (int o = 0; o < KS; ++o) {
          if (o == zr) continue;
          const uint32_t rbase =
              dsmem_map(smem_u32(recv), (uint32_t)o) + (uint32_t)((zr < o ? zr : zr - 1) * c_n * kBM * 4);
#pragma unroll 1
          for (int g = half; g < c_n / 8; g += kParts) {
            uint32_t r[8];
            tmem_ld8(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(o * c_n + 8 * g), r);
            tmem_ld_wait();
#pragma unroll
            for (int k = 0; k < 8; ++k)
              dsmem_st_f32(rbase + (uint32_t)(((8 * g + k) * kBM + sub * 32 + lane) * 4), __uint_as_float(r[k]));
          }
        }
      cluster_sync();
    }
    if (!all_ok) {
      if (t == 0) atomicOr(a.err, 2);
    } else {
      // view geometry in registers (the loop reads no kernel parameters)
      float* const ext = a.out.ext;
      const int64_t ext_ch = (int64_t)ph_l * a.cout + ch_l;
      const int32_t f_rows = a.out.f32.rows, f_p16 = a.out.f32.chans / 4;
      const int32_t l_rows0 = a.out.lp[0].rows, l_rows1 = a.out.lp[1].rows;
      const int32_t l_p16_0 = a.out.lp[0].chans / 8, l_p16_1 = a.out.lp[1].chans / 8;
      const int32_t l_mir0 = a.out.lp[0].rows - a.out.lp[0].pre, l_mir1 = a.out.lp[1].rows - a.out.lp[1].pre;
      const bool l_bf16 = (l_rows0 ? a.out.lp[0].dtype : a.out.lp[1].dtype) == kDtBF16;
      const bool has_skip = a.has_skip != 0;
      char* const f_base = arena + (int64_t)ch_l * 4;
      char* const l_base = arena + (int64_t)ch_l * 2;
      const uint32_t stg_base = smem_u32(sB);
      const int stg_q0 = (rsub * 32 + 8 * (lane & 3)) >> 2;  // this lane's first 16-byte chunk of a column
#pragma unroll 1
      for (int cb = c_lo + 32 * rpart; cb < c_lo + c_n; cb += cstep) {
        if (n0 + cb >= N) break;  // uniform over the warp
        const int cl = cb + lane;
        const int64_t eb = col_ext[cl];
        const uint32_t fo = col_off[cl], lo0 = col_off[BN + cl], lo1 = col_off[2 * BN + cl];
        const uint32_t lm0 = col_mir[cl], lm1 = col_mir[BN + cl];
        const int32_t fr = col_row[cl], lr0 = col_row[BN + cl], lr1 = col_row[2 * BN + cl];
        const uint32_t so_cur = so_next;
        const int32_t sr_cur = sr_next;
        if (has_skip && cb + cstep < c_lo + c_n) {
          so_next = col_off[3 * BN + cl + cstep];
          sr_next = col_row[3 * BN + cl + cstep];
        }
#pragma unroll 1
        for (int g = half; g < 4; g += kParts) {
          if (n0 + cb + 8 * g >= N) break;  // uniform
          uint32_t r[8];
          tmem_ld8(tmem + ((uint32_t)(sub * 32) << 16) + acc_col + (uint32_t)(cb + 8 * g), r);
          tmem_ld_wait();
          if (KS > 1) {
            // own partial (TMEM) and the received ones, summed in the order z = 0, 1, ...
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float* rc = recv + (cb - c_lo + 8 * g + k) * kBM + sub * 32 + lane;
              const float own = __uint_as_float(r[k]);
              float acc = 0.f;
#pragma unroll
              for (int z = 0; z < 4; ++z)
                if (z < KS) acc += z == zr ? own : rc[(z < zr ? z : z - 1) * c_n * kBM];
              r[k] = __float_as_uint(acc);
            }
          }
          // turn: row-per-lane values in, 8-channel column slices out
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 8; ++k) tw[k * 32 + lane] = fmaf(__uint_as_float(r[k]), sc, bi);
          __syncwarp();
          const float4 v0 = *reinterpret_cast<const float4*>(tw + kk * 32 + 8 * (lane & 3));
          const float4 v1 = *reinterpret_cast<const float4*>(tw + kk * 32 + 8 * (lane & 3) + 4);
          float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
          if (staged) {
            const int c = cb + 8 * g + kk;  // tile column (fused units: c_lo = 0)
            const uint32_t rb = stg_base + (uint32_t)(c * stg_rows * 4);
            const float4 s0 = ld_shared_v4(rb + (uint32_t)((stg_q0 ^ (c & 1)) << 4));
            const float4 s1 = ld_shared_v4(rb + (uint32_t)(((stg_q0 + 1) ^ (c & 1)) << 4));
            x[0] += s0.x; x[1] += s0.y; x[2] += s0.z; x[3] += s0.w;
            x[4] += s1.x; x[5] += s1.y; x[6] += s1.z; x[7] += s1.w;
          } else if (has_skip) {
            x[0] += sk0.x; x[1] += sk0.y; x[2] += sk0.z; x[3] += sk0.w;
            x[4] += sk1.x; x[5] += sk1.y; x[6] += sk1.z; x[7] += sk1.w;
            // the next group's residual loads overlap this group's stores
            if (g + kParts < 4)
              load_skip(cb, g + kParts, so_cur, sr_cur);
            else if (cb + cstep < c_lo + c_n && n0 + cb + cstep < N)
              load_skip(cb + cstep, half, so_next, sr_next);
          }
          const int src = 8 * g + kk;  // table lane of this lane's column
          const bool ok = vok && n0 + cb + src < N;
          if (ext) {
            const int64_t e = shfl64(eb, src) + ext_ch;
            if (ok)
#pragma unroll
              for (int i = 0; i < 8; ++i) st_global_f32(ext + e + i, x[i]);
          }
          if (f_rows) {
            uint32_t o = __shfl_sync(0xffffffffu, fo, src);
            const int32_t rw = __shfl_sync(0xffffffffu, fr, src);
            if (phased) o = phase_off(o, rw, f_rows, f_p16);
            char* pa = f_base + (uint64_t)o * 16;
            if (ok) {
              st_global_v4(pa, make_uint4(__float_as_uint(x[0]), __float_as_uint(x[1]), __float_as_uint(x[2]),
                                          __float_as_uint(x[3])));
              st_global_v4(pa + 16, make_uint4(__float_as_uint(x[4]), __float_as_uint(x[5]),
                                               __float_as_uint(x[6]), __float_as_uint(x[7])));
            }
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int32_t rows = q ? l_rows1 : l_rows0;
            if (!rows) continue;
            float y[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) y[i] = q ? leaky(x[i]) : x[i];
            const uint4 pk = make_uint4(pack2(y[0], y[1], l_bf16), pack2(y[2], y[3], l_bf16),
                                        pack2(y[4], y[5], l_bf16), pack2(y[6], y[7], l_bf16));
            uint32_t o = __shfl_sync(0xffffffffu, q ? lo1 : lo0, src);
            uint32_t om = __shfl_sync(0xffffffffu, q ? lm1 : lm0, src);
            if (phased) {
              const int32_t rw = __shfl_sync(0xffffffffu, q ? lr1 : lr0, src);
              const int32_t p16 = q ? l_p16_1 : l_p16_0;
              const int32_t d = rw + ph_l >= rows ? ph_l - rows : ph_l;
              o += (uint32_t)(d * p16);
              om = rw + d >= (q ? l_mir1 : l_mir0) ? o - (uint32_t)(rows * p16) : ~0u;
            }
            if (ok) st_global_v4(l_base + (uint64_t)o * 16, pk);
            if (ok && om != ~0u) st_global_v4(l_base + (uint64_t)om * 16, pk);  // mirrored tail
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, L::kTmemCols);
}

template <int BN, int STAGES, bool FUSE, int EW, bool SPLIT = false, int MT = 1>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, int ks, cudaStream_t st) {
  static bool configured = false;
  using L = TcLayout<BN, STAGES, FUSE, EW, SPLIT, MT>;
  constexpr int bytes = L::kBytes;
  static_assert(bytes <= 232448, "shared memory per CTA");
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<BN, STAGES, FUSE, EW, SPLIT, MT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  const int mtiles = (a.M + kBM - 1) / kBM;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)mtiles, (unsigned)ks);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(L::kThreads);
  cfg.dynamicSmemBytes = (size_t)bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 1;
  attr[1].val.clusterDim.y = (unsigned)MT;
  attr[1].val.clusterDim.z = (unsigned)ks;
  cfg.attrs = attr;
  cfg.numAttrs = (ks > 1 || MT > 1) ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_conv_tc<BN, STAGES, FUSE, EW, SPLIT, MT>, ta, tb, a);
}

}  // namespace

int tc_tile_n(int64_t n_cols, int m_tiles) {
  return ((n_cols + 255) / 256) * m_tiles >= 152 ? 256 : 128;
}

cudaError_t launch_conv_tc(const void* tmap_t, const void* tmap_b, const TcArgs& a, int bn,
                           cudaStream_t st) {
  const int64_t N = (int64_t)a.batch.count * a.ncols;
  if (N <= 0) return cudaSuccess;
  const CUtensorMap& ta = *reinterpret_cast<const CUtensorMap*>(tmap_t);
  const CUtensorMap& tb = *reinterpret_cast<const CUtensorMap*>(tmap_b);
  const int ks = a.ksplit > 1 ? a.ksplit : 1;
  if (a.k2 > 0) {
    // fused residual unit: 128-column tiles, no split; one M tile (M <= 128),
    // or two as a cluster exchanging the intermediate (M <= 256, one wave)
    if (ks != 1) return cudaErrorInvalidValue;
    if (a.M > kBM) {
      if (a.M > 2 * kBM || a.k2 > 4 || !a.deep_ok) return cudaErrorInvalidValue;
      return launch_bn<128, 4, true, 16, false, 2>(ta, tb, a, 1, st);
    }
    if (a.k2 > 2) return cudaErrorInvalidValue;
    if (a.deep_ok && (N + 127) / 128 <= 148) return launch_bn<128, 4, true, 16>(ta, tb, a, 1, st);
    return launch_bn<128, 2, true, 8>(ta, tb, a, 1, st);
  }
  if (bn == 256 && ks == 1) return launch_bn<256, 4, false, 8>(ta, tb, a, 1, st);
  const int64_t ctas = (N + 127) / 128 * ((a.M + kBM - 1) / kBM) * ks;
  if (ks > 1) {
    if (ks > 4) return cudaErrorInvalidValue;
    return launch_bn<128, 4, false, 16, true>(ta, tb, a, ks, st);
  }
  if (ctas <= 148 && a.deep_ok) return launch_bn<128, 6, false, 16>(ta, tb, a, 1, st);
  return launch_bn<128, 3, false, 8>(ta, tb, a, 1, st);
}

}  // namespace cc
