// Host-side model and plan structures of the runtime (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/cachedconv.h"
#include "cc_internal.h"

namespace cc {

cc_status fail(cc_status code, const char* fmt, ...);

// Analysis and storage plan of one node of the reconfigured model.
struct NodePlan {
  cc_node_desc d{};
  int64_t rnum = 1, rden = 1;  // frames per input frame
  int32_t u = 0;               // frames per model step
  int64_t D = 0;               // cumulated delay (own frames), section 3.1
  int32_t Da = 0;              // Eq. 2 extra delay (strided conv)
  int32_t A[3] = {0, 0, 0};    // Eq. 3 alignment per input (merges)
  int32_t hist_need = 0;       // cached frames this layer reads before its window
  int32_t keep = 0;            // frames of this node's output kept for consumers
  std::vector<int> consumers;
  // output views: 0 FP32, 1 low precision as computed, 2 low precision after
  // LeakyReLU; keep_view = history kept for the consumers of that view
  bool has_ring = false;
  bool used_view[3] = {false, false, false};
  int32_t keep_view[3] = {0, 0, 0};
  Ring view[3]{};
  int32_t engine = 0;  // 0: FP32 FFMA kernels, 1: tcgen05 tensor cores
  // residual add folded into this conv's epilogue
  int32_t fused_add = -1, fused_skip = -1, fused_skip_A = 0;
  bool fused = false;  // (add) computed by its producer's epilogue
  // packed GEMM view
  int32_t M = 0, Kt = 0, taps = 0, phases = 1;
  float* dA = nullptr;
  float* dbias = nullptr;
  // tensor-core operand: low-precision [Mpad][Kt], per-row scale, TMA map
  int32_t Mpad = 0;
  void* dA_lp = nullptr;
  void* dA_tiled = nullptr;
  float* dscale = nullptr;
  alignas(64) unsigned char tmap[128] = {};   // weights
  alignas(64) unsigned char tmapB[128] = {};  // input view as arena rows
  // input view as [slot][pre + R][C], boxes of 64 x 2^i rows x 2^(7-i) slots
  alignas(64) unsigned char tmapT[8][128] = {};
  bool tmapT_ok[8] = {};
  int32_t in_rows_per_slot = 0, in_row_off = 0;
  int32_t ksplit = 1;  // tensor-core split-K factor, fixed per layer (batch-independent numerics)
  int32_t unit_next = -1;  // this conv and the 1x1 conv (node unit_next) run as one launch
  // sibling group: stride-1 tensor-core convs sharing their input, computed by
  // one contraction of the leader; members' FP32 views share one ring
  int32_t group_leader = -1;
  int32_t choff = 0;                 // (member) first channel in the group's ring
  std::vector<int> group;            // (leader) members, leader first
  int32_t group_taps = 0, group_hist = 0;  // (leader) merged window
  bool unit_fused = false;  // (1x1 conv) computed by its producer's fused launch
  bool no_split = false;    // a unit the model could fuse but runs unfused: unsplit K, as if fused
  std::map<int64_t, int32_t> tile_n;  // autotuned N tile by launch width (columns), 0: heuristic
};

struct TimingRec {
  int node;
  cudaEvent_t start, stop;
};

struct Model {
  int32_t dtype = CC_F32;
  int32_t lp_dtype = kDtBF16;  // element type of low-precision views
  int32_t max_streams = 0, max_steps = 1, noise = 1;
  int32_t fuse_units = 1;  // residual units (k-wide conv -> 1x1 conv) as one tensor-core launch
  int32_t merge_siblings = 1;  // tensor-core convs sharing their input as one contraction
  int32_t in_per_step = 1;
  std::vector<NodePlan> nodes;
  size_t slot_bytes = 0, state_bytes = 0, weight_bytes = 0;
  char* arena = nullptr;
  int32_t* err = nullptr;  // device error word (bounded waits that gave up)
  int32_t* withhold = nullptr;  // failure-detection test counter (launches left to withhold a copy)
  uint64_t wait_ns = 2000000000ull;  // limit of every device-side pipeline wait
  int64_t* counters = nullptr;
  uint64_t* seeds = nullptr;
  float* in_manip = nullptr;  // [max_streams][3][input channels]: per-slot scale, bias, noise amplitude
  std::mutex mu;
  std::vector<int32_t> free_slots;
  std::vector<cc_stream*> live_streams;  // destroyed with the model
  // batch slot lists, one per CUDA stream (batches on different CUDA
  // streams may run concurrently): device list, pinned staging, the event
  // guarding the staging, and the last list uploaded
  struct SlotList {
    int32_t* d = nullptr;
    int32_t* h = nullptr;
    cudaEvent_t uploaded = nullptr;
    std::vector<int32_t> cache;
    bool valid = false;
  };
  std::map<cudaStream_t, SlotList> slot_lists;
  int32_t* batch_slots = nullptr;  // the default CUDA stream's list (allocated at creation)
  // host I/O staging, one pair of device buffers per CUDA stream (calls on
  // different CUDA streams may overlap on the GPU)
  struct Staging {
    float* in = nullptr;
    float* out = nullptr;
    size_t in_bytes = 0, out_bytes = 0;
  };
  std::map<cudaStream_t, Staging> stagings;
  // launch chains of host-buffer calls, captured once per (streams, steps,
  // device slot list, staging) and replayed: they read and write only the
  // staging buffers (dropped when a staging grows or the tile shapes change)
  struct ChainGraph {
    int32_t count, steps;
    const int32_t* d_slots;
    const float *in, *out;
    cudaGraphExec_t exec;
  };
  std::vector<ChainGraph> chain_graphs;
  cudaStream_t capture_stream = nullptr;
  void drop_chain_graphs(const float* in = nullptr, const float* out = nullptr);
  // ragged-batch / FIFO staging: one row of whole steps per stream
  float* rag_in = nullptr;
  float* rag_out = nullptr;
  size_t rag_in_bytes = 0, rag_out_bytes = 0;
  // per-node timing
  bool timing_on = false;
  std::vector<TimingRec> timing_recs;
  std::vector<cudaEvent_t> event_pool;
  size_t event_pool_used = 0;

  int32_t force_tile_n = 0;  // autotuning: every tensor-core layer uses this N tile
  int32_t last_chain_launches = 0;  // kernels the most recent launch chain enqueued
  // the cached state as ring regions (a stream's snapshot copies only these rows)
  struct StateRegion {
    int64_t off;        // byte offset of ring row 0 in a slot
    int32_t rows, pre;  // ring rows R; mirrored rows before row 0 (low-precision views)
    int32_t row_bytes;  // bytes per row (a multiple of 4)
    int32_t keep;       // rows of history kept: times t0 - keep .. t0 - 1
    int32_t u;          // frames per model step of the ring
  };
  std::vector<StateRegion> state_regions;
  StateRegion* d_state_regions = nullptr;  // device copy
  size_t snapshot_bytes = 0;               // 16 (counter, seed) + every region's kept rows

  ~Model();
  int32_t tile_n_for(const NodePlan& p, int64_t n_cols) const;
  cc_status autotune(const int32_t* d_slots, int32_t count, const float* in, int64_t in_stride, float* out,
                     int64_t out_stride, cudaStream_t st);
  Batch batch_for(const int32_t* d_slots, int32_t count) const;
  cc_status process(const int32_t* d_slots, int32_t count, const float* in, int64_t in_stride,
                    int64_t n_in, float* out, int64_t out_stride, int64_t n_out, cudaStream_t st);
  cc_status run_chain(const Batch& b, const float* in, int64_t in_stride, float* out,
                      int64_t out_stride, int32_t steps, cudaStream_t st);
  cc_status ensure_staging(int32_t count, cudaStream_t st, Staging** sg);
  cudaError_t take_event(cudaEvent_t* ev);
};

}  // namespace cc

// A stream: one arena slot of cache state (section 2.2), its noise seed, and,
// in FIFO mode (buffers that need not be whole model steps), the input frames
// still short of a step and the output frames produced but not yet delivered.
struct cc_stream {
  cc::Model* model;
  int32_t slot;
  uint64_t seed;
  int32_t* d_slot;
  bool manip_set = false;  // a non-identity input manipulation is in place
  bool fifo = false;
  int64_t prefill = 0;     // zero output frames queued when FIFO mode was switched on
  float* in_q = nullptr;   // [in_per_step][in channels] device: pending input frames
  int64_t in_frames = 0;
  float* out_q[2] = {nullptr, nullptr};  // [out_cap][out channels] device, ping-pong
  int64_t out_frames = 0, out_cap = 0;
  int32_t out_cur = 0;
};

namespace cc {
// FIFO and ragged-batch processing (cc_batch.cu)
cc_status process_ragged(Model* m, cc_stream* const* streams, const float* const* in, const int64_t* n_in,
                         float* const* out, const int64_t* n_out, int32_t count, cudaStream_t st);
cc_status upload_slot_list(Model* m, const std::vector<int32_t>& slots, cudaStream_t st, const int32_t** d_list);
void free_fifo(cc_stream* s);
}  // namespace cc
