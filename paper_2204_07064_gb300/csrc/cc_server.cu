// Serving loop: continuous batching of many real-time streams of one model.
//
// Clients submit requests (a stream, some input frames, a number of output
// frames wanted) from any thread.  A scheduler thread repeatedly takes every
// stream that has a request still waiting for output and at least one model
// step of input buffered, and advances all of them by one step in a single
// launch chain (the streams' caches stay resident in their arena slots; the
// batch is a device list of slots).  Streams that arrive while a batch is on
// the GPU join the next one.  Output beyond what a request asked for waits in
// the stream's FIFO for its next request, so requests shorter than a model
// step (e.g. 512-sample buffers of a decoder that emits 2048 samples per
// step) are served from the FIFO.  Each batch size is padded to a bucket with
// a scratch slot and its launch chain is replayed from a CUDA graph; the tile
// shapes of each bucket come from the model's autotuner.  For large batches
// the per-stream host work (gathering inputs, handing outputs to requests) is
// split across worker threads, and an output goes straight into the waiting
// request's buffer when the stream's FIFO is empty.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/cachedconv.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {
extern thread_local std::string g_last_error;
int32_t stream_slot(const cc_stream* s);
Model* stream_model(const cc_stream* s);
}  // namespace cc

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// batches of at least kParallelMin streams split their host work across up
// to kWorkers threads
constexpr int32_t kParallelMin = 1024;
constexpr int32_t kWorkers = 8;

struct Request {
  float* out;
  int64_t n_out;  // output frames still owed
  int64_t done_frames = 0;
  uint64_t tag;
  int64_t submit_ns;
};

// Contiguous float FIFO (block copies; the consumed prefix is dropped lazily).
struct FloatFifo {
  std::vector<float> buf;
  size_t head = 0;
  size_t size() const { return buf.size() - head; }
  void push(const float* p, size_t n) { buf.insert(buf.end(), p, p + n); }
  void pop(float* dst, size_t n) {
    std::memcpy(dst, buf.data() + head, n * sizeof(float));
    head += n;
    if (head == buf.size()) {
      buf.clear();
      head = 0;
    } else if (head > 4096 && head * 2 > buf.size()) {
      buf.erase(buf.begin(), buf.begin() + head);
      head = 0;
    }
  }
};

// Worker threads kept for the life of a server: run(fn) calls fn(k) on
// worker k = 1..size()-1 and on the caller as worker 0, and returns when all
// are done.
class Pool {
 public:
  explicit Pool(int32_t n) {
    for (int32_t k = 1; k < n; ++k) th_.emplace_back([this, k] { work(k); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(m_);
      quit_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  int32_t size() const { return (int32_t)th_.size() + 1; }
  void run(const std::function<void(int32_t)>& fn) {
    {
      std::lock_guard<std::mutex> g(m_);
      fn_ = &fn;
      pending_ = (int32_t)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    fn(0);
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return pending_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work(int32_t k) {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(int32_t)>* f = nullptr;
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (quit_) return;
        f = fn_;
      }
      (*f)(k);
      std::lock_guard<std::mutex> g(m_);
      if (--pending_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, done_;
  const std::function<void(int32_t)>* fn_ = nullptr;
  int32_t pending_ = 0;
  uint64_t gen_ = 0;
  bool quit_ = false;
};

struct StreamQueue {
  bool queued = false;  // listed in the server's ready list
  FloatFifo in;   // buffered input (interleaved frames)
  FloatFifo out;  // produced, not yet delivered output
  std::deque<Request> reqs;
  int64_t owed = 0;  // output frames requested but not delivered
};

struct Completion {
  uint64_t tag;
  int64_t submit_ns, step_ns, done_ns;  // step_ns: start of the GPU step that completed it
};

}  // namespace

struct cc_server {
  cc::Model* m = nullptr;
  cc_server_config cfg{};
  int32_t cin = 0, cout = 0, in_step = 0, out_step = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  // device / pinned staging
  float *d_in = nullptr, *d_out = nullptr, *h_in = nullptr, *h_out = nullptr;
  int32_t *d_slots = nullptr, *h_slots = nullptr;
  int32_t* d_scratch_slots = nullptr;  // cap copies of the scratch slot
  int32_t cap = 0;  // padded batch capacity
  cc_stream* scratch = nullptr;
  std::map<int32_t, cudaGraphExec_t> graphs;
  std::unordered_set<int32_t> tuned;
  // client state
  std::mutex mu;
  std::condition_variable cv, idle_cv;
  std::unordered_map<cc_stream*, StreamQueue> q;
  std::unordered_set<cc_stream*> in_flight;
  std::vector<Completion> done;
  bool stop = false;
  cc_status error = CC_OK;
  std::string error_msg;
  std::thread th;
  bool preparing = false;  // cc_server_prepare owns the GPU side
  std::vector<StreamQueue*> sq_ptr;                   // the batch's queues
  // streams that may need a step (submitted to, or served, since they were
  // last batched); an entry counts only while its queue's `queued` is set,
  // so removed or re-listed streams are skipped
  std::vector<cc_stream*> ready_list, cand;
  std::unique_ptr<Pool> pool;
  std::vector<Completion> part_done[kWorkers];        // completions found by workers 1..
  // statistics
  int64_t batches = 0, stream_steps = 0, gpu_ns = 0, max_batch_seen = 0;
  int64_t setups = 0, setup_ns = 0;  // first batches of a bucket: tuning, warm-up, graph capture

  int32_t bucket(int32_t count) const {
    const int32_t g = cfg.bucket > 0 ? cfg.bucket : 32;
    int32_t b = (count + g - 1) / g * g;
    return std::min(b, cap);
  }
  bool needs_step(const StreamQueue& s) const {
    return s.owed * cout > (int64_t)s.out.size() && (int64_t)s.in.size() >= (int64_t)in_step * cin;
  }
  void mark(cc_stream* st, StreamQueue& s) {
    if (!s.queued && needs_step(s)) {
      s.queued = true;
      ready_list.push_back(st);
    }
  }
  // fn(begin, end, worker) over [0, n) in contiguous parts, on the pool's
  // threads from kParallelMin items on
  template <typename F>
  void parallel_parts(int32_t n, F fn) {
    const int32_t w = (n < kParallelMin || !pool) ? 1 : pool->size();
    if (w == 1) {
      fn(0, n, 0);
      return;
    }
    const int32_t per = (n + w - 1) / w;
    pool->run([&](int32_t k) {
      const int32_t a = k * per, b = std::min(n, a + per);
      if (a < b) fn(a, b, k);
    });
  }
  void serve_fifo(StreamQueue& s, int64_t t, int64_t t_step) { serve_fifo(s, t, t_step, done); }
  void serve_fifo(StreamQueue& s, int64_t t, int64_t t_step, std::vector<Completion>& out_done) {
    while (!s.reqs.empty()) {
      Request& r = s.reqs.front();
      const int64_t avail = (int64_t)s.out.size() / cout;
      const int64_t take = std::min(avail, r.n_out - r.done_frames);
      if (take > 0) s.out.pop(r.out + r.done_frames * cout, (size_t)(take * cout));
      r.done_frames += take;
      s.owed -= take;
      if (r.done_frames < r.n_out) break;
      out_done.push_back(Completion{r.tag, r.submit_ns, t_step, t});
      s.reqs.pop_front();
    }
  }
  // A step's output of one stream: straight into the waiting requests'
  // buffers while the FIFO is empty, the rest into the FIFO.
  void deliver(StreamQueue& s, const float* src, size_t n, int64_t t, int64_t t_step, std::vector<Completion>& out_done) {
    size_t off = 0;
    if (s.out.size() == 0) {
      while (off < n && !s.reqs.empty()) {
        Request& r = s.reqs.front();
        const int64_t take = std::min<int64_t>((int64_t)((n - off) / cout), r.n_out - r.done_frames);
        if (take > 0) std::memcpy(r.out + r.done_frames * cout, src + off, (size_t)take * cout * sizeof(float));
        off += (size_t)take * cout;
        r.done_frames += take;
        s.owed -= take;
        if (r.done_frames < r.n_out) break;
        out_done.push_back(Completion{r.tag, r.submit_ns, t_step, t});
        s.reqs.pop_front();
      }
    }
    if (off < n) s.out.push(src + off, n - off);
    serve_fifo(s, t, t_step, out_done);
  }
  bool ready(int32_t padded) const {
    return (!cfg.autotune || tuned.count(padded)) && (!cfg.use_graphs || graphs.count(padded));
  }
  cc_status setup(int32_t padded);
  cc_status gpu_step(int32_t count, int32_t padded);
  void loop();
};

namespace {

#define SRV_CUDA(call)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return cc::fail(CC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// First batch of a bucket: tune tile shapes and warm the kernels up on a batch
// made of the scratch slot only (its rings are never read back), then capture
// the bucket's launch chain.
cc_status cc_server::setup(int32_t padded) {
  const int64_t is = (int64_t)in_step * cin, os = (int64_t)out_step * cout;
  {
    const cc::Batch scratch_batch = m->batch_for(d_scratch_slots, padded);
    if (cfg.autotune && !tuned.count(padded)) {
      cc_status s = m->autotune(d_scratch_slots, padded, d_in, is, d_out, os, st);
      if (s) return s;
      tuned.insert(padded);
    } else {
      cc_status s = m->run_chain(scratch_batch, d_in, is, d_out, os, 1, st);
      if (s) return s;
    }
    SRV_CUDA(cudaStreamSynchronize(st));
    if (cfg.use_graphs) {
      // capture the chain of this bucket; it reads the slot list from d_slots
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      SRV_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cc_status s = m->run_chain(m->batch_for(d_slots, padded), d_in, is, d_out, os, 1, st);
      cudaError_t ce = cudaStreamEndCapture(st, &g);
      if (s) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (ce != cudaSuccess) return cc::fail(CC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return cc::fail(CC_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
      graphs.emplace(padded, ge);
    }
  }
  return CC_OK;
}

cc_status cc_server::gpu_step(int32_t count, int32_t padded) {
  const int64_t is = (int64_t)in_step * cin, os = (int64_t)out_step * cout;
  SRV_CUDA(cudaMemcpyAsync(d_slots, h_slots, sizeof(int32_t) * padded, cudaMemcpyHostToDevice, st));
  SRV_CUDA(cudaMemcpyAsync(d_in, h_in, sizeof(float) * (size_t)padded * is, cudaMemcpyHostToDevice, st));
  if (cfg.use_graphs) {
    SRV_CUDA(cudaGraphLaunch(graphs.at(padded), st));
  } else {
    cc_status s = m->run_chain(m->batch_for(d_slots, padded), d_in, is, d_out, os, 1, st);
    if (s) return s;
  }
  SRV_CUDA(cudaMemcpyAsync(h_out, d_out, sizeof(float) * (size_t)count * os, cudaMemcpyDeviceToHost, st));
  SRV_CUDA(cudaStreamSynchronize(st));
  return CC_OK;
}

void cc_server::loop() {
  {
    const int32_t hw = (int32_t)std::max(1u, std::thread::hardware_concurrency());
    const int32_t w = std::min(kWorkers, std::max(1, hw / 2));
    if (w > 1) pool.reset(new Pool(w));
  }
  std::vector<cc_stream*> batch;
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    if (preparing) {
      cv.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    // every stream with a request waiting and a step of input (from the
    // ready list), oldest request first
    batch.clear();
    cand.swap(ready_list);
    for (cc_stream* st : cand) {
      auto it = q.find(st);
      if (it == q.end() || !it->second.queued) continue;
      it->second.queued = false;
      if (needs_step(it->second)) batch.push_back(st);
    }
    cand.clear();
    if ((int32_t)batch.size() > cfg.max_batch) {
      std::nth_element(batch.begin(), batch.begin() + cfg.max_batch, batch.end(),
                       [&](cc_stream* x, cc_stream* y) {
                         return q[x].reqs.front().submit_ns < q[y].reqs.front().submit_ns;
                       });
      for (size_t k = cfg.max_batch; k < batch.size(); ++k) {
        q[batch[k]].queued = true;
        ready_list.push_back(batch[k]);
      }
      batch.resize(cfg.max_batch);
    }
    if (batch.empty()) {
      cv.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    const int32_t count = (int32_t)batch.size();
    const int32_t padded = bucket(count);
    const size_t step_in = (size_t)in_step * cin;
    // (the scheduler holds the lock: nothing else touches the queues)
    sq_ptr.resize(count);
    for (int32_t i = 0; i < count; ++i) {
      sq_ptr[i] = &q[batch[i]];
      in_flight.insert(batch[i]);
    }
    parallel_parts(count, [&](int32_t a, int32_t b, int32_t) {
      for (int32_t i = a; i < b; ++i) {
        h_slots[i] = cc::stream_slot(batch[i]);
        sq_ptr[i]->in.pop(h_in + i * step_in, step_in);
      }
    });
    const int32_t sslot = cc::stream_slot(scratch);
    for (int32_t i = count; i < padded; ++i) {
      h_slots[i] = sslot;
      std::memset(h_in + i * step_in, 0, step_in * sizeof(float));
    }
    lk.unlock();
    int64_t t_setup = 0;
    cc_status s = CC_OK;
    if (!ready(padded)) {
      const int64_t a = now_ns();
      s = setup(padded);
      t_setup = now_ns() - a;
    }
    const int64_t t0 = now_ns();
    if (!s) s = gpu_step(count, padded);
    const int64_t t1 = now_ns();
    lk.lock();
    if (s) {
      error = s;
      error_msg = cc::g_last_error;
      stop = true;
      in_flight.clear();
      idle_cv.notify_all();
      break;
    }
    ++batches;
    stream_steps += count;
    gpu_ns += t1 - t0;
    if (t_setup) {
      ++setups;
      setup_ns += t_setup;
    }
    max_batch_seen = std::max<int64_t>(max_batch_seen, count);
    const size_t step_out = (size_t)out_step * cout;
    // (streams removed meanwhile waited for this batch: every queue is there)
    parallel_parts(count, [&](int32_t a, int32_t b, int32_t w) {
      std::vector<Completion>& mine = w == 0 ? done : part_done[w];
      for (int32_t i = a; i < b; ++i) deliver(*sq_ptr[i], h_out + i * step_out, step_out, t1, t0, mine);
    });
    for (int32_t w = 1; w < kWorkers; ++w) {
      done.insert(done.end(), part_done[w].begin(), part_done[w].end());
      part_done[w].clear();
    }
    for (int32_t i = 0; i < count; ++i) mark(batch[i], *sq_ptr[i]);
    in_flight.clear();
    idle_cv.notify_all();
  }
}

extern "C" {

cc_status cc_server_create(cc_model* model, const cc_server_config* config, cc_server** out) {
  using cc::fail;
  if (!model || !config || !out) return fail(CC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (config->max_batch <= 0 || config->max_batch > m->max_streams)
    return fail(CC_ERR_INVALID_ARG, "max_batch must be in [1, max_streams]");
  auto* s = new cc_server();
  s->m = m;
  s->cfg = *config;
  s->cin = m->nodes.front().d.c_in;
  s->cout = m->nodes.back().d.c_out;
  s->in_step = m->in_per_step;
  s->out_step = m->nodes.back().u;
  const int32_t g = config->bucket > 0 ? config->bucket : 32;
  s->cap = (config->max_batch + g - 1) / g * g;
  cc_status r = CC_OK;
  auto cleanup = [&]() {
    if (s->scratch) cc_stream_destroy(s->scratch);
    if (s->d_in) cudaFree(s->d_in);
    if (s->d_out) cudaFree(s->d_out);
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->h_in) cudaFreeHost(s->h_in);
    if (s->h_out) cudaFreeHost(s->h_out);
    if (s->h_slots) cudaFreeHost(s->h_slots);
    if (s->d_scratch_slots) cudaFree(s->d_scratch_slots);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
  };
  // the scratch slot pads batches to their bucket (its contents are never read back)
  r = cc_stream_create(model, 0, nullptr, &s->scratch);
  if (r) {
    cleanup();
    return fail(CC_ERR_NO_MEMORY, "the server needs one free stream slot for padding: %s",
                cc::g_last_error.c_str());
  }
  const size_t nin = (size_t)s->cap * s->in_step * s->cin, nout = (size_t)s->cap * s->out_step * s->cout;
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&s->d_in, nin * 4) != cudaSuccess || cudaMalloc(&s->d_out, nout * 4) != cudaSuccess ||
      cudaMalloc(&s->d_slots, sizeof(int32_t) * s->cap) != cudaSuccess ||
      cudaMallocHost(&s->h_in, nin * 4) != cudaSuccess || cudaMallocHost(&s->h_out, nout * 4) != cudaSuccess ||
      cudaMallocHost(&s->h_slots, sizeof(int32_t) * s->cap) != cudaSuccess ||
      cudaMalloc(&s->d_scratch_slots, sizeof(int32_t) * s->cap) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(CC_ERR_NO_MEMORY, "server buffers");
  }
  {
    std::vector<int32_t> fill(s->cap, cc::stream_slot(s->scratch));
    if (cudaMemcpy(s->d_scratch_slots, fill.data(), sizeof(int32_t) * s->cap, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cleanup();
      return fail(CC_ERR_CUDA, "server scratch slot list upload failed");
    }
  }
  cudaGetDevice(&s->device);
  s->th = std::thread([s]() {
    cudaSetDevice(s->device);
    s->loop();
  });
  *out = s;
  return CC_OK;
}

cc_status cc_server_destroy(cc_server* s) {
  if (!s) return cc::fail(CC_ERR_INVALID_ARG, "null server");
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  cc_stream_destroy(s->scratch);
  cudaFree(s->d_in);
  cudaFree(s->d_out);
  cudaFree(s->d_slots);
  cudaFreeHost(s->h_in);
  cudaFreeHost(s->h_out);
  cudaFreeHost(s->h_slots);
  cudaFree(s->d_scratch_slots);
  cudaStreamDestroy(s->st);
  delete s;
  return CC_OK;
}

cc_status cc_server_submit(cc_server* s, int32_t count, cc_stream* const* streams, const float* const* in,
                           const int64_t* n_in, float* const* out, const int64_t* n_out,
                           const uint64_t* tags) {
  using cc::fail;
  if (!s || count < 0 || (count && (!streams || !n_in || !n_out || !tags)))
    return fail(CC_ERR_INVALID_ARG, "null argument");
  const int64_t t = now_ns();
  std::lock_guard<std::mutex> g(s->mu);
  if (s->error) return fail(s->error, "server stopped: %s", s->error_msg.c_str());
  for (int32_t i = 0; i < count; ++i) {
    cc_stream* st = streams[i];
    if (!st || cc::stream_model(st) != s->m) return fail(CC_ERR_INVALID_ARG, "request %d: stream of another model", i);
    if (n_in[i] < 0 || n_out[i] < 0) return fail(CC_ERR_INVALID_ARG, "request %d: negative length", i);
    if ((n_in[i] && (!in || !in[i])) || (n_out[i] && (!out || !out[i])))
      return fail(CC_ERR_INVALID_ARG, "request %d: null buffer", i);
  }
  for (int32_t i = 0; i < count; ++i) {
    StreamQueue& q = s->q[streams[i]];
    if (n_in[i]) q.in.push(in[i], (size_t)(n_in[i] * s->cin));
    q.owed += n_out[i];
    q.reqs.push_back(Request{n_out[i] ? out[i] : nullptr, n_out[i], 0, tags[i], t});
    s->serve_fifo(q, t, t);
    s->mark(streams[i], q);
  }
  s->cv.notify_one();
  return CC_OK;
}

cc_status cc_server_poll(cc_server* s, int32_t max, uint64_t* tags, int64_t* submit_ns, int64_t* step_ns,
                         int64_t* done_ns, int32_t* got) {
  if (!s || !got || max < 0) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  const int32_t n = std::min<int32_t>(max, (int32_t)s->done.size());
  for (int32_t i = 0; i < n; ++i) {
    if (tags) tags[i] = s->done[i].tag;
    if (submit_ns) submit_ns[i] = s->done[i].submit_ns;
    if (step_ns) step_ns[i] = s->done[i].step_ns;
    if (done_ns) done_ns[i] = s->done[i].done_ns;
  }
  s->done.erase(s->done.begin(), s->done.begin() + n);
  *got = n;
  if (s->error) return cc::fail(s->error, "server stopped: %s", s->error_msg.c_str());
  return CC_OK;
}

cc_status cc_server_remove(cc_server* s, cc_stream* stream) {
  if (!s || !stream) return cc::fail(CC_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  s->idle_cv.wait(lk, [&] { return !s->in_flight.count(stream) || s->stop; });
  s->q.erase(stream);
  return CC_OK;
}

cc_status cc_server_stats(cc_server* s, int64_t* batches, int64_t* stream_steps, int64_t* gpu_ns,
                          int64_t* max_batch, int64_t* setups, int64_t* setup_ns) {
  if (!s) return cc::fail(CC_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> g(s->mu);
  if (batches) *batches = s->batches;
  if (stream_steps) *stream_steps = s->stream_steps;
  if (gpu_ns) *gpu_ns = s->gpu_ns;
  if (max_batch) *max_batch = s->max_batch_seen;
  if (setups) *setups = s->setups;
  if (setup_ns) *setup_ns = s->setup_ns;
  return CC_OK;
}

cc_status cc_server_prepare(cc_server* s, int32_t max_count) {
  if (!s) return cc::fail(CC_ERR_INVALID_ARG, "null server");
  if (max_count < 1 || max_count > s->cfg.max_batch)
    return cc::fail(CC_ERR_INVALID_ARG, "max_count must be in [1, max_batch]");
  std::unique_lock<std::mutex> lk(s->mu);
  // wait for the batch on the GPU, then hold the scheduler off
  s->idle_cv.wait(lk, [&] { return s->in_flight.empty() || s->stop; });
  if (s->error) return cc::fail(s->error, "server stopped: %s", s->error_msg.c_str());
  s->preparing = true;
  lk.unlock();
  cc_status r = CC_OK;
  int64_t n = 0, ns = 0;
  for (int32_t c = 1; c <= max_count && r == CC_OK;) {
    const int32_t padded = s->bucket(c);
    if (!s->ready(padded)) {
      const int64_t a = now_ns();
      r = s->setup(padded);
      ns += now_ns() - a;
      ++n;
    }
    if (padded >= s->cap) break;
    c = padded + 1;
  }
  lk.lock();
  s->preparing = false;
  s->setups += n;
  s->setup_ns += ns;
  s->cv.notify_one();
  return r;
}

}  // extern "C"
