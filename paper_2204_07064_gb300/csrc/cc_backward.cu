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

#include <cstring>
#include <vector>

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

struct BwdView {
  Ring r;          // FP32 view geometry (same offsets in both arenas)
  int64_t t0;      // absolute time of the chunk's first frame at this node
};

__device__ __forceinline__ float* adj_ptr(char* adj, int64_t slot_bytes, int32_t slot, const Ring& r,
                                          int64_t t) {
  return reinterpret_cast<float*>(adj + (int64_t)slot * slot_bytes + r.off) + ring_row(t, r.rows) * r.chans;
}

__device__ __forceinline__ const float* fwd_ptr(const Batch& b, int32_t s, const Ring& r, int64_t t) {
  return reinterpret_cast<const float*>(slot_base(b, s) + r.off) + ring_row(t, r.rows) * r.chans;
}

__device__ __forceinline__ int64_t chunk_t0(const Batch& b, int32_t s, int32_t u, int32_t steps) {
  return (steps_of(b, s) - steps) * (int64_t)u;
}

// Zero the adjoint rows of times [t0 - keep, t0 + n - keep) for every stream.
__global__ void k_adj_clear(Batch b, char* adj, Ring r, int32_t keep, int32_t n, int32_t steps) {
  const int64_t total = (int64_t)b.count * n * r.chans;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i % r.chans);
    const int64_t q = i / r.chans;
    const int32_t j = (int32_t)(q % n);
    const int32_t s = (int32_t)(q / n);
    const int64_t t = chunk_t0(b, s, r.u, steps) - keep + j;
    adj_ptr(adj, b.slot_bytes, b.slots[s], r, t)[c] = 0.f;
  }
}

struct BwdConv {
  const float* W;   // trained layout: conv [cout][cin][K], convt [cin][cout][K]
  int32_t op;       // CC_OP_CONV / CC_OP_CONVT
  int32_t cin, cout, K, S, dil, hist, act;
  int32_t n_in, n_out;  // frames of this chunk per stream, input / output rate
  Ring x;               // forward FP32 view of the input (pre-activation values)
  int32_t u_in, u_out;
  Ring gy;              // adjoint ring of the output node (rows == 0: gy_ext)
  const float* gy_ext;  // caller's output gradient, stream s at gy_ext + s*gy_stride
  int64_t gy_stride;
  float* dW;  // trained layout accumulators
  float* db;
  int32_t steps;
  Batch b;
  char* adj;
};

__device__ __forceinline__ float load_gy(const BwdConv& a, int32_t s, int64_t t0_out, int32_t o, int32_t n) {
  if (a.gy.rows == 0) return a.gy_ext[(int64_t)s * a.gy_stride + (int64_t)o * a.cout + n];
  return adj_ptr(a.adj, a.b.slot_bytes, a.b.slots[s], a.gy, t0_out + o)[n];
}

// dL/dx for input frames i in [-hist, n_in) of the chunk (history included),
// times the LeakyReLU derivative, accumulated into the input's adjoint ring.
// Only the chunk's own output frames contribute: later outputs were handled
// by later chunks, which already scattered into these rows.
__global__ void k_bwd_data(BwdConv a) {
  const int32_t span = a.hist + a.n_in;
  const int64_t total = (int64_t)a.b.count * span * a.cin;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = (int32_t)(idx % a.cin);
    const int64_t q = idx / a.cin;
    const int32_t i = (int32_t)(q % span) - a.hist;
    const int32_t s = (int32_t)(q / span);
    const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
    float acc = 0.f;
    if (a.op == CC_OP_CONV) {
      for (int32_t k = 0; k < a.K; ++k) {
        const int32_t jj = i + a.hist - k * a.dil;
        if (jj < 0 || jj % a.S) continue;
        const int32_t o = jj / a.S;
        if (o >= a.n_out) continue;
        for (int32_t n = 0; n < a.cout; ++n)
          acc = fmaf(a.W[((int64_t)n * a.cin + m) * a.K + k], load_gy(a, s, t0_out, o, n), acc);
      }
    } else {
      const int32_t T = a.K / a.S;
      for (int32_t jj = 0; jj < T; ++jj) {
        const int32_t qq = i + jj;  // output block fed by input frame i through tap jj
        if (qq < 0 || qq >= a.n_in) continue;
        for (int32_t ph = 0; ph < a.S; ++ph) {
          const int32_t o = qq * a.S + ph;
          const float* wrow = a.W + (int64_t)m * a.cout * a.K + ph + jj * a.S;
          for (int32_t n = 0; n < a.cout; ++n) acc = fmaf(wrow[(int64_t)n * a.K], load_gy(a, s, t0_out, o, n), acc);
        }
      }
    }
    const int64_t t = t0_in + i;
    if (a.act) {
      const float xpre = fwd_ptr(a.b, s, a.x, t)[m];
      acc *= xpre >= 0.f ? 1.f : kLeakySlope;
    }
    adj_ptr(a.adj, a.b.slot_bytes, a.b.slots[s], a.x, t)[m] += acc;
  }
}

// dL/dW and dL/db of this chunk, added to the accumulators; one thread per
// weight, reduction over every stream and output frame of the chunk.
__global__ void k_bwd_weight(BwdConv a) {
  const int64_t total = (int64_t)a.cout * a.cin * a.K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f, bacc = 0.f;
    if (a.op == CC_OP_CONV) {
      // idx -> (n, k, m), m fastest for coalesced input reads
      const int32_t m = (int32_t)(idx % a.cin);
      const int64_t r = idx / a.cin;
      const int32_t k = (int32_t)(r % a.K);
      const int32_t n = (int32_t)(r / a.K);
      const bool do_bias = a.db && m == 0 && k == 0;
      for (int32_t s = 0; s < a.b.count; ++s) {
        const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
        for (int32_t o = 0; o < a.n_out; ++o) {
          const float g = load_gy(a, s, t0_out, o, n);
          const float xin = activate(fwd_ptr(a.b, s, a.x, t0_in + (int64_t)o * a.S + k * a.dil - a.hist)[m], a.act);
          acc = fmaf(g, xin, acc);
          if (do_bias) bacc += g;
        }
      }
      a.dW[((int64_t)n * a.cin + m) * a.K + k] += acc;
      if (do_bias) a.db[n] += bacc;
    } else {
      // idx -> (n, kk, m): W[m][n][kk], kk = ph + jj*S
      const int32_t m = (int32_t)(idx % a.cin);
      const int64_t r = idx / a.cin;
      const int32_t kk = (int32_t)(r % a.K);
      const int32_t n = (int32_t)(r / a.K);
      const int32_t ph = kk % a.S, jj = kk / a.S;
      const bool do_bias = a.db && m == 0 && kk == 0;
      for (int32_t s = 0; s < a.b.count; ++s) {
        const int64_t t0_in = chunk_t0(a.b, s, a.u_in, a.steps), t0_out = chunk_t0(a.b, s, a.u_out, a.steps);
        for (int32_t qq = 0; qq < a.n_in; ++qq) {
          const float g = load_gy(a, s, t0_out, qq * a.S + ph, n);
          const float xin = activate(fwd_ptr(a.b, s, a.x, t0_in + qq - jj)[m], a.act);
          acc = fmaf(g, xin, acc);
        }
        if (do_bias)
          for (int32_t o = 0; o < a.n_out; ++o) bacc += load_gy(a, s, t0_out, o, n);
      }
      a.dW[((int64_t)m * a.cout + n) * a.K + kk] += acc;
      if (do_bias) a.db[n] += bacc;
    }
  }
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
};

__global__ void k_bwd_merge(BwdMerge a) {
  const int64_t total = (int64_t)a.b.count * a.n * a.chans;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(idx % a.chans);
    const int64_t q = idx / a.chans;
    const int32_t j = (int32_t)(q % a.n);
    const int32_t s = (int32_t)(q / a.n);
    const int64_t t = chunk_t0(a.b, s, a.u, a.steps) + j;
    const float g = a.gy.rows ? adj_ptr(a.adj, a.b.slot_bytes, a.b.slots[s], a.gy, t)[c]
                              : a.gy_ext[(int64_t)s * a.gy_stride + (int64_t)j * a.chans + c];
    if (a.op == CC_OP_ADD) {
      for (int k = 0; k < a.nin; ++k)
        if (a.gin[k].rows) adj_ptr(a.adj, a.b.slot_bytes, a.b.slots[s], a.gin[k], t - a.A[k])[c] += g;
    } else {
      const float w = fwd_ptr(a.b, s, a.in[0], t - a.A[0])[c];
      const float am = fwd_ptr(a.b, s, a.in[1], t - a.A[1])[c];
      const float nz = fwd_ptr(a.b, s, a.in[2], t - a.A[2])[c];
      const float th = tanhf(w), sa = 1.f / (1.f + expf(-am)), sn = 1.f / (1.f + expf(-nz));
      float u = 0.f;
      if (a.noise) u = noise_uniform(a.b.seeds[a.b.slots[s]], t - a.delay, c, a.chans);
      const float gw = g * (1.f - th * th) * sa, ga = g * th * sa * (1.f - sa), gn = g * u * sn * (1.f - sn);
      const float gs[3] = {gw, ga, gn};
      for (int k = 0; k < 3; ++k)
        if (a.gin[k].rows) adj_ptr(a.adj, a.b.slot_bytes, a.b.slots[s], a.gin[k], t - a.A[k])[c] += gs[k];
    }
  }
}

__global__ void k_adj_out(Batch b, char* adj, Ring r, int32_t n, int32_t steps, float* gx, int64_t stride) {
  const int64_t total = (int64_t)b.count * n * r.chans;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i % r.chans);
    const int64_t q = i / r.chans;
    const int32_t j = (int32_t)(q % n);
    const int32_t s = (int32_t)(q / n);
    gx[(int64_t)s * stride + (int64_t)j * r.chans + c] =
        adj_ptr(adj, b.slot_bytes, b.slots[s], r, chunk_t0(b, s, r.u, steps) + j)[c];
  }
}

int grid_of(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

// ===========================================================================
struct cc_grads {
  cc::Model* m = nullptr;
  char* adj = nullptr;
  std::vector<float*> dW, db;
  std::vector<size_t> nW;
  std::vector<float*> dW_dev_trained;  // trained-layout FP32 weights per node (for backward data)
  int32_t* d_slots = nullptr;
  int32_t* h_slots = nullptr;
  cudaEvent_t upload_done = nullptr;
};

extern "C" {

cc_status cc_grads_create(cc_model* model, const float* const* weights, cc_grads** out) {
  using cc::fail;
  if (!model || !out || !weights) return fail(CC_ERR_INVALID_ARG, "null argument");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (m->dtype != CC_F32) return fail(CC_ERR_STATE, "the backward pass runs on FP32 models");
  if (m->max_streams == 0) return fail(CC_ERR_STATE, "plan-only model");
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
  g->dW_dev_trained.assign(n, nullptr);
  auto bad = [&](const char* what) {
    cudaGetLastError();
    for (size_t i = 0; i < n; ++i) {
      if (g->dW[i]) cudaFree(g->dW[i]);
      if (g->db[i]) cudaFree(g->db[i]);
      if (g->dW_dev_trained[i]) cudaFree(g->dW_dev_trained[i]);
    }
    if (g->adj) cudaFree(g->adj);
    if (g->d_slots) cudaFree(g->d_slots);
    if (g->h_slots) cudaFreeHost(g->h_slots);
    delete g;
    return fail(CC_ERR_NO_MEMORY, "gradient buffers: %s", what);
  };
  if (cudaMalloc(&g->adj, m->slot_bytes * (size_t)m->max_streams) != cudaSuccess) return bad("adjoint arena");
  if (cudaMemset(g->adj, 0, m->slot_bytes * (size_t)m->max_streams) != cudaSuccess) return bad("adjoint arena");
  if (cudaMalloc(&g->d_slots, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
      cudaMallocHost(&g->h_slots, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->upload_done, cudaEventDisableTiming) != cudaSuccess)
    return bad("batch list");
  for (size_t i = 0; i < n; ++i) {
    const cc_node_desc& d = m->nodes[i].d;
    if (d.op != CC_OP_CONV && d.op != CC_OP_CONVT) continue;
    g->nW[i] = (size_t)d.c_in * d.c_out * d.kernel;
    if (cudaMalloc(&g->dW[i], g->nW[i] * 4) != cudaSuccess ||
        cudaMalloc(&g->dW_dev_trained[i], g->nW[i] * 4) != cudaSuccess)
      return bad("weight gradient");
    if (cudaMemcpy(g->dW_dev_trained[i], weights[i], g->nW[i] * 4, cudaMemcpyHostToDevice) != cudaSuccess)
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
    if (g->dW_dev_trained[i]) cudaFree(g->dW_dev_trained[i]);
  }
  cudaFree(g->adj);
  cudaFree(g->d_slots);
  cudaFreeHost(g->h_slots);
  cudaEventDestroy(g->upload_done);
  delete g;
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
  if (dw && cudaMemcpy(dw, g->dW[node], g->nW[node] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cc::fail(CC_ERR_CUDA, "copy failed");
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
    const cudaError_t e = cudaMemsetAsync(g->adj + (size_t)cc::stream_slot(streams[i]) * g->m->slot_bytes, 0,
                                          g->m->slot_bytes, st);
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
  // batch list (the pinned staging may still feed the previous upload)
  BW_CUDA(cudaEventSynchronize(g->upload_done));
  for (int32_t i = 0; i < count; ++i) {
    if (!streams[i] || cc::stream_model(streams[i]) != m) return fail(CC_ERR_INVALID_ARG, "stream %d", i);
    if (cc::stream_manipulated(streams[i]))
      return fail(CC_ERR_STATE, "stream %d has an input manipulation; the backward does not differentiate it", i);
    g->h_slots[i] = cc::stream_slot(streams[i]);
  }
  BW_CUDA(cudaMemcpyAsync(g->d_slots, g->h_slots, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
  BW_CUDA(cudaEventRecord(g->upload_done, st));
  const cc::Batch b = m->batch_for(g->d_slots, count);
  // 1. recompute this chunk's forward from the restored state; its output is
  //    not needed (grad_x doubles as scratch only if the shapes agree, so use
  //    the model's staging buffers)
  cc_status s = m->ensure_staging(count);
  if (s) return s;
  s = m->run_chain(b, x, x_stride, m->stage_out, (int64_t)steps * m->nodes.back().u * m->nodes.back().d.c_out,
                   steps, st);
  if (s) return s;
  // 2. clear the adjoint rows no later chunk could have written
  const int n = (int)m->nodes.size();
  for (int i = 0; i < n; ++i) {
    const cc::NodePlan& p = m->nodes[i];
    if (!p.view[0].rows) continue;
    const int32_t nn = p.u * steps;
    k_adj_clear<<<grid_of((int64_t)count * nn * p.d.c_out), 256, 0, st>>>(b, g->adj, p.view[0], p.keep_view[0], nn,
                                                                          steps);
    BW_CUDA(cudaGetLastError());
  }
  // 3. nodes in reverse order
  auto gy_ring = [&](int wi) -> cc::Ring { return wi == n - 1 ? cc::Ring{} : m->nodes[wi].view[0]; };
  for (int i = n - 1; i >= 1; --i) {
    const cc::NodePlan& p = m->nodes[i];
    const cc_node_desc& d = p.d;
    if (d.op == CC_OP_CONV || d.op == CC_OP_CONVT) {
      const int wi = p.fused_add >= 0 ? p.fused_add : i;
      if (wi != n - 1 && !m->nodes[wi].view[0].rows) continue;  // dead branch: zero adjoint
      const cc::NodePlan& src = m->nodes[d.inputs[0]];
      BwdConv a{};
      a.W = g->dW_dev_trained[i];
      a.op = d.op;
      a.cin = d.c_in;
      a.cout = d.c_out;
      a.K = d.kernel;
      a.S = d.stride;
      a.dil = d.op == CC_OP_CONV ? d.dilation : 1;
      a.hist = p.hist_need;
      a.act = d.act_in;
      a.n_in = src.u * steps;
      a.n_out = m->nodes[wi].u * steps;
      a.x = src.view[0];
      a.u_in = src.u;
      a.u_out = m->nodes[wi].u;
      a.gy = gy_ring(wi);
      a.gy_ext = grad_y;
      a.gy_stride = gy_stride;
      a.dW = g->dW[i];
      a.db = g->db[i];
      a.steps = steps;
      a.b = b;
      a.adj = g->adj;
      k_bwd_data<<<grid_of((int64_t)count * (a.hist + a.n_in) * a.cin), 256, 0, st>>>(a);
      BW_CUDA(cudaGetLastError());
      k_bwd_weight<<<grid_of((int64_t)a.cout * a.cin * a.K), 256, 0, st>>>(a);
      BW_CUDA(cudaGetLastError());
    } else if (d.op == CC_OP_ADD || d.op == CC_OP_HEADS) {
      if (i != n - 1 && !p.view[0].rows) continue;  // dead branch
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
        a.gin[k] = into_conv ? cc::Ring{} : m->nodes[src].view[0];
        a.A[k] = p.A[k];
      }
      a.delay = p.D;
      a.noise = m->noise;
      a.b = b;
      a.adj = g->adj;
      k_bwd_merge<<<grid_of((int64_t)count * a.n * a.chans), 256, 0, st>>>(a);
      BW_CUDA(cudaGetLastError());
    }
  }
  // 4. the input adjoint of this chunk's frames
  if (grad_x) {
    const cc::NodePlan& p0 = m->nodes[0];
    k_adj_out<<<grid_of((int64_t)count * p0.u * steps * p0.d.c_out), 256, 0, st>>>(b, g->adj, p0.view[0],
                                                                                   p0.u * steps, steps, grad_x,
                                                                                   gx_stride);
    BW_CUDA(cudaGetLastError());
  }
#undef BW_CUDA
  return CC_OK;
}

cc_status cc_stream_snapshot(cc_stream* s, void* dev, size_t bytes, void* cuda_stream) {
  if (!s || !dev) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  cc::Model* m = cc::stream_model(s);
  if (bytes != m->slot_bytes + 16) return cc::fail(CC_ERR_INVALID_ARG, "snapshot size must be %zu", m->slot_bytes + 16);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int32_t slot = cc::stream_slot(s);
  char* d = static_cast<char*>(dev);
  if (cudaMemcpyAsync(d, m->counters + slot, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d + 8, m->seeds + slot, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d + 16, m->arena + (size_t)slot * m->slot_bytes, m->slot_bytes, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return cc::fail(CC_ERR_CUDA, "snapshot copy failed");
  return CC_OK;
}

cc_status cc_stream_restore(cc_stream* s, const void* dev, size_t bytes, void* cuda_stream) {
  if (!s || !dev) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  cc::Model* m = cc::stream_model(s);
  if (bytes != m->slot_bytes + 16) return cc::fail(CC_ERR_INVALID_ARG, "snapshot size must be %zu", m->slot_bytes + 16);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int32_t slot = cc::stream_slot(s);
  const char* d = static_cast<const char*>(dev);
  if (cudaMemcpyAsync(m->counters + slot, d, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->seeds + slot, d + 8, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->arena + (size_t)slot * m->slot_bytes, d + 16, m->slot_bytes, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return cc::fail(CC_ERR_CUDA, "restore copy failed");
  return CC_OK;
}

}  // extern "C"
