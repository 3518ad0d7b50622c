// Ragged batches and buffers that are not whole model steps.
//
// The paper's DSP call processes whatever buffer the host hands it (section 1,
// section 5.1).  A model step is the smallest input length that keeps every
// strided layer aligned (section 3.1): for the RAVE-like decoder one latent
// frame (2048 output samples), for an encoder 2048 input samples.  Two
// entry points relax the whole-step rule:
//   - cc_process_batch advances any number of distinct streams, each by its
//     own number of whole steps (a ragged batch): streams with equal step
//     counts share one launch chain;
//   - a stream in FIFO mode accepts any input length and any output length.
//     Input short of a whole step waits in the stream's input queue; a step
//     runs as soon as its input is complete; output frames wait in the
//     stream's output queue until a call asks for them.  The output queue
//     starts with `prefill` zero frames, which is the extra latency the
//     caller accepts: for a model that consumes whole steps of S input frames
//     and a caller that hands over b < S frames per call and wants b' output
//     frames back at once, prefill = out_per_step - gcd(b', out_per_step)
//     (out_per_step - b' when b' divides it) makes every call servable, and
//     the stream's delay grows by exactly that.
// Every buffer goes through a per-model device staging area laid out as one
// row of whole steps per stream, so that the launch chains keep their
// strided layout; copies are cudaMemcpyAsync on the caller's CUDA stream
// (host or device buffers alike).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/cachedconv.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {

#define CCB_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(CC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void free_fifo(cc_stream* s) {
  if (s->in_q) cudaFree(s->in_q);
  for (auto& q : s->out_q)
    if (q) cudaFree(q);
  s->in_q = nullptr;
  s->out_q[0] = s->out_q[1] = nullptr;
  s->fifo = false;
  s->in_frames = s->out_frames = s->out_cap = s->prefill = 0;
  s->out_cur = 0;
}

static cc_status grow(float** buf, size_t* have, size_t need) {
  if (need <= *have) return CC_OK;
  if (*buf) cudaFree(*buf);  // synchronises: no copy still reads it
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(CC_ERR_NO_MEMORY, "staging buffer of %zu bytes", need);
  }
  *have = need;
  return CC_OK;
}

// Both output queues of a FIFO stream hold at least `frames` frames; the
// live one keeps its contents.
static cc_status ensure_out_cap(cc_stream* s, int64_t frames, int32_t cout, cudaStream_t st) {
  if (frames <= s->out_cap) return CC_OK;
  const int64_t cap = std::max<int64_t>(frames, 2 * s->out_cap);
  float* fresh[2] = {nullptr, nullptr};
  for (auto& f : fresh)
    if (cudaMalloc(&f, sizeof(float) * cap * cout) != cudaSuccess) {
      cudaGetLastError();
      for (auto& g : fresh)
        if (g) cudaFree(g);
      return fail(CC_ERR_NO_MEMORY, "FIFO output queue of %lld frames", (long long)cap);
    }
  if (s->out_frames)
    CCB_CUDA(cudaMemcpyAsync(fresh[0], s->out_q[s->out_cur], sizeof(float) * s->out_frames * cout,
                             cudaMemcpyDeviceToDevice, st));
  CCB_CUDA(cudaStreamSynchronize(st));
  for (auto& q : s->out_q)
    if (q) cudaFree(q);
  s->out_q[0] = fresh[0];
  s->out_q[1] = fresh[1];
  s->out_cur = 0;
  s->out_cap = cap;
  return CC_OK;
}

static cc_status copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes) CCB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
  return CC_OK;
}

cc_status process_ragged(Model* m, cc_stream* const* ss, const float* const* in, const int64_t* n_in,
                         float* const* out, const int64_t* n_out, int32_t count, cudaStream_t st) {
  if (count > m->max_streams) return fail(CC_ERR_INVALID_ARG, "batch larger than max_streams");
  const int32_t cin = m->nodes.front().d.c_in, cout = m->nodes.back().d.c_out;
  const int64_t ips = m->in_per_step, ops = m->nodes.back().u;
  std::vector<int64_t> k(count);
  std::vector<int32_t> slots(count);
  for (int32_t i = 0; i < count; ++i) {
    cc_stream* s = ss[i];
    if (!s || s->model != m) return fail(CC_ERR_INVALID_ARG, "stream %d not of this model", i);
    if (n_in[i] < 0 || n_out[i] < 0) return fail(CC_ERR_INVALID_ARG, "stream %d: negative length", i);
    if ((n_in[i] && (!in || !in[i])) || (n_out[i] && (!out || !out[i])))
      return fail(CC_ERR_INVALID_ARG, "stream %d: null buffer", i);
    slots[i] = s->slot;
    if (s->fifo) {
      k[i] = (s->in_frames + n_in[i]) / ips;
      const int64_t avail = s->out_frames + k[i] * ops;
      if (n_out[i] > avail)
        return fail(CC_ERR_BAD_LENGTH,
                    "stream %d (FIFO mode) asks for %lld output frames; %lld are queued or due from this "
                    "call's input",
                    i, (long long)n_out[i], (long long)avail);
    } else {
      if (n_in[i] % ips != 0)
        return fail(CC_ERR_BAD_LENGTH, "stream %d: n_in %lld is not a multiple of the model step (%lld frames)",
                    i, (long long)n_in[i], (long long)ips);
      k[i] = n_in[i] / ips;
      if (n_out[i] != k[i] * ops)
        return fail(CC_ERR_BAD_LENGTH, "stream %d: n_out %lld != %lld steps x %lld output frames", i,
                    (long long)n_out[i], (long long)k[i], (long long)ops);
    }
  }
  {
    std::vector<int32_t> sorted = slots;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(CC_ERR_INVALID_ARG, "a stream appears twice in one batch");
  }
  // staging rows: streams with steps to run, most steps first
  std::vector<int32_t> order;
  for (int32_t i = 0; i < count; ++i)
    if (k[i] > 0) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return k[a] > k[b]; });
  const int32_t rows = (int32_t)order.size();
  const int64_t kmax = rows ? k[order[0]] : 0;
  const int64_t rs_in = kmax * ips * cin, rs_out = kmax * ops * cout;  // floats per row
  if (rows) {
    cc_status r = grow(&m->rag_in, &m->rag_in_bytes, sizeof(float) * rs_in * rows);
    if (!r) r = grow(&m->rag_out, &m->rag_out_bytes, sizeof(float) * rs_out * rows);
    if (r) return r;
  }
  const size_t fin = sizeof(float) * cin, fout = sizeof(float) * cout;
  // inputs: whole steps into the staging rows; FIFO remainders into the input queues
  std::vector<int32_t> row_of(count, -1);
  for (int32_t r = 0; r < rows; ++r) row_of[order[r]] = r;
  for (int32_t i = 0; i < count; ++i) {
    cc_stream* s = ss[i];
    cc_status c = CC_OK;
    if (!s->fifo) {
      if (k[i]) c = copy(m->rag_in + row_of[i] * rs_in, in[i], fin * n_in[i], st);
    } else if (k[i] == 0) {
      c = copy(s->in_q + s->in_frames * cin, in[i], fin * n_in[i], st);
      s->in_frames += n_in[i];
    } else {
      float* row = m->rag_in + row_of[i] * rs_in;
      const int64_t take = k[i] * ips - s->in_frames;  // frames of this call's input in the steps
      c = copy(row, s->in_q, fin * s->in_frames, st);
      if (!c) c = copy(row + s->in_frames * cin, in[i], fin * take, st);
      const int64_t rest = n_in[i] - take;
      if (!c) c = copy(s->in_q, in[i] + take * cin, fin * rest, st);
      s->in_frames = rest;
    }
    if (c) return c;
  }
  // one launch chain per group of equal step counts (at most max_steps steps each)
  if (rows) {
    std::vector<int32_t> row_slots(rows);
    for (int32_t r = 0; r < rows; ++r) row_slots[r] = slots[order[r]];
    const int32_t* d_list = nullptr;
    cc_status c = upload_slot_list(m, row_slots, st, &d_list);
    if (c) return c;
    for (int32_t g0 = 0; g0 < rows;) {
      int32_t g1 = g0;
      while (g1 < rows && k[order[g1]] == k[order[g0]]) ++g1;
      const int64_t kg = k[order[g0]];
      const Batch b = m->batch_for(d_list + g0, g1 - g0);
      for (int64_t done = 0; done < kg; done += m->max_steps) {
        const int32_t steps = (int32_t)std::min<int64_t>(m->max_steps, kg - done);
        c = m->run_chain(b, m->rag_in + g0 * rs_in + done * ips * cin, rs_in,
                         m->rag_out + g0 * rs_out + done * ops * cout, rs_out, steps, st);
        if (c) return c;
      }
      g0 = g1;
    }
  }
  // outputs: whole rows to the caller; FIFO streams are served from their
  // queue first, the rest of the new frames is queued
  for (int32_t i = 0; i < count; ++i) {
    cc_stream* s = ss[i];
    const float* row = k[i] ? m->rag_out + row_of[i] * rs_out : nullptr;
    cc_status c = CC_OK;
    if (!s->fifo) {
      if (k[i]) c = copy(out[i], row, fout * n_out[i], st);
      if (c) return c;
      continue;
    }
    const int64_t produced = k[i] * ops;
    const int64_t a = std::min(n_out[i], s->out_frames);  // from the queue
    const int64_t b = n_out[i] - a;                       // from this call's steps
    const int64_t left = s->out_frames - a + produced - b;
    c = ensure_out_cap(s, left, cout, st);
    if (c) return c;
    float* cur = s->out_q[s->out_cur];
    float* nxt = s->out_q[1 - s->out_cur];
    c = copy(out[i], cur, fout * a, st);
    if (!c) c = copy(out[i] + a * cout, row, fout * b, st);
    if (!c && n_out[i]) {  // the undelivered frames move to the front of the other queue
      c = copy(nxt, cur + a * cout, fout * (s->out_frames - a), st);
      if (!c) c = copy(nxt + (s->out_frames - a) * cout, row + b * cout, fout * (produced - b), st);
      s->out_cur = 1 - s->out_cur;
    } else if (!c && produced) {  // nothing delivered: append
      c = copy(cur + s->out_frames * cout, row, fout * produced, st);
    }
    if (c) return c;
    s->out_frames = left;
  }
  return CC_OK;
}

}  // namespace cc

using cc::fail;

extern "C" {

cc_status cc_stream_set_fifo(cc_stream* s, int32_t enable, int64_t prefill_frames, void* cuda_stream) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  cc::Model* m = s->model;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  CCB_CUDA(cudaStreamSynchronize(st));
  cc::free_fifo(s);
  if (!enable) return CC_OK;
  if (prefill_frames < 0) return fail(CC_ERR_INVALID_ARG, "negative prefill");
  const int32_t cin = m->nodes.front().d.c_in, cout = m->nodes.back().d.c_out;
  const int64_t ops = m->nodes.back().u;
  if (cudaMalloc(&s->in_q, sizeof(float) * m->in_per_step * cin) != cudaSuccess) {
    cudaGetLastError();
    s->in_q = nullptr;
    return fail(CC_ERR_NO_MEMORY, "FIFO input queue");
  }
  s->fifo = true;
  s->prefill = prefill_frames;
  cc_status r = cc::ensure_out_cap(s, std::max<int64_t>(prefill_frames + ops, 2 * ops), cout, st);
  if (r) {
    cc::free_fifo(s);
    return r;
  }
  s->out_frames = prefill_frames;
  if (prefill_frames) CCB_CUDA(cudaMemsetAsync(s->out_q[0], 0, sizeof(float) * prefill_frames * cout, st));
  return CC_OK;
}

cc_status cc_stream_delay(const cc_stream* s, int64_t* out_frames) {
  if (!s || !out_frames) return fail(CC_ERR_INVALID_ARG, "null argument");
  *out_frames = s->model->nodes.back().D + (s->fifo ? s->prefill : 0);
  return CC_OK;
}

cc_status cc_stream_fifo_state(const cc_stream* s, int64_t* in_frames, int64_t* out_frames) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  if (in_frames) *in_frames = s->fifo ? s->in_frames : 0;
  if (out_frames) *out_frames = s->fifo ? s->out_frames : 0;
  return CC_OK;
}

}  // extern "C"
