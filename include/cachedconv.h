/*
 * cachedconv.h -- C ABI of the GB300 (sm_103a) streamed-convolution library.
 *
 * Buffer-by-buffer inference of a non-causal 1-D convolutional audio model
 * after post-training causal reconfiguration (Caillon & Esling, "Streamable
 * neural audio synthesis with non-causal convolutions", DAFx-22):
 *   - cached padding: every convolution keeps the last N input frames of the
 *     previous buffer and uses them instead of zero left padding (section 2.2,
 *     Fig. 1);
 *   - right padding is moved to the left after training, which delays the
 *     layer's output (section 3);
 *   - strided convolutions receive an extra input delay D_a (Eq. 2,
 *     section 3.1); transposed convolutions only delay their output;
 *   - parallel branches are re-aligned by extra delays A_i (Eq. 3, section 3.2).
 * The calls follow the paper's statement of the problem: a model is built from
 * its layer list and weights, each audio stream owns a cache state, each DSP
 * call processes one buffer (section 1, section 5.1), and the total latency
 * is queried so that it can be compensated (section 4.2, section 4.3).
 *
 * Conventions for every entry point:
 *   - Signals are float32, channels-last ("interleaved"): element (t, c) of a
 *     buffer with C channels is at index t*C + c.
 *   - Pointers to signal buffers may be device or host memory (detected per
 *     call).  Host buffers are staged through device memory inside the call;
 *     the call is asynchronous on `cuda_stream` in both cases, so the caller
 *     synchronises that stream before reading a host output buffer.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - The caller owns every buffer it passes.  The library copies weights in;
 *     a model owns its packed weights, its state arena and its streams' slots.
 *   - Errors are returned as negative cc_status values, never by aborting; a
 *     thread-local message is available from cc_last_error().
 *   - A stream must not be processed concurrently with itself; different
 *     streams may be processed concurrently on different CUDA streams only if
 *     they are not in the same batch call.  Calls on one model come from one
 *     host thread at a time (its host-side plan, staging and graph caches are
 *     not locked); the serving scheduler (cc_server_*) is the exception and
 *     documents its own rules.
 */
#ifndef CACHEDCONV_H
#define CACHEDCONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cc_status;
#define CC_OK 0
#define CC_ERR_INVALID_ARG (-1) /* null pointer, bad enum, out-of-range size */
#define CC_ERR_BAD_GRAPH (-2)   /* layer list not a valid streamable DAG       */
#define CC_ERR_BAD_LENGTH (-3)  /* buffer length not a multiple of a model step */
#define CC_ERR_NO_MEMORY (-4)   /* arena full (admission) or allocation failed */
#define CC_ERR_CUDA (-5)        /* a CUDA runtime call failed                   */
#define CC_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up           */
#define CC_ERR_STATE (-7)       /* object used in the wrong state               */

typedef enum {
  CC_OP_INPUT = 0, /* the model input (exactly one, node 0)                          */
  CC_OP_CONV = 1,  /* Conv1d, Eq. 1 with stride, dilation, trained pads L/R          */
  CC_OP_CONVT = 2, /* ConvTranspose1d, stride S, kernel K (K % S == 0), left crop p  */
  CC_OP_ADD = 3,   /* sum of two branches (residual), aligned by Eq. 3               */
  CC_OP_HEADS = 4  /* tanh(in0)*sigmoid(in1) + sigmoid(in2)*u, branches aligned by Eq. 3,
                      u = SplitMix64 noise in [-1,1) keyed on the aligned frame index */
} cc_op;

typedef enum { CC_ACT_NONE = 0, CC_ACT_LEAKY = 1 /* LeakyReLU, slope 0.2, on the node input */ } cc_act;

typedef enum {
  CC_F32 = 0,  /* FP32 storage, FP32 FFMA contractions                                   */
  CC_BF16 = 1, /* BF16 operands on tensor cores (tcgen05), FP32 accumulation            */
  CC_F16 = 2   /* FP16 operands on tensor cores (tcgen05), FP32 accumulation            */
} cc_dtype;
/* In the BF16/FP16 modes a conv or convT runs on the tensor cores when
 * c_in % 64 == 0 and c_out % 8 == 0.  It multiplies its activated input
 * rounded to that type (nearest even) by its weights rounded row by row: each
 * GEMM row (a conv's output channel over input channels and taps; a convT's
 * output channel and output phase over input channels and that phase's taps)
 * is scaled to max |w| = 1 before rounding, and the FP32 scale is applied to
 * the FP32 accumulator.  Every other layer, and every value kept for merges,
 * stays FP32. */

/* One layer of the trained (non-causal) model, in topological order. */
typedef struct {
  int32_t op;        /* cc_op                                                      */
  int32_t n_inputs;  /* 0 (input), 1 (conv/convt), 2 (add), 3 (heads)              */
  int32_t inputs[3]; /* producer node indices, each < this node's index           */
  int32_t c_in, c_out;
  int32_t kernel, stride, dilation;
  int32_t pad_left, pad_right; /* trained zero padding, in input frames (conv)    */
  int32_t crop;                /* trained left crop p of the full ConvT output;
                                  the trained right crop is K - S - p             */
  int32_t act_in;              /* cc_act applied to the node's input              */
  int32_t has_bias;
} cc_node_desc;

typedef struct {
  int32_t compute;            /* cc_dtype                                             */
  int32_t max_streams;        /* number of per-stream state slots in the arena (with
                                 arena_bytes > 0: an upper bound, 0 = none); both 0
                                 builds a plan only (analysis queries, no device
                                 memory, no weights needed; streams cannot be created) */
  int32_t max_steps_per_call; /* model steps one launch chain covers (longer buffers are
                                 split); sizes the per-slot scratch rows              */
  int32_t noise;              /* 1: heads add sigmoid(in2)*u; 0: u = 0 (section 4.2)  */
  int32_t flags;              /* CC_FLAG_* bits (0: defaults)                          */
  int64_t arena_bytes;        /* > 0: device memory budget of the stream arena; the
                                 model holds as many stream slots as fit
                                 (floor(arena_bytes / slot bytes), capped by
                                 max_streams if that is > 0), so streams are admitted
                                 by cache memory; NO_MEMORY if not even one fits     */
  int64_t wait_limit_ns;      /* limit of every device-side pipeline wait (0: 2 s);
                                 a wait that runs out records TIMEOUT (see
                                 cc_model_device_status) instead of hanging          */
} cc_model_config;

/* cc_model_config.flags: launch each convolution of a residual unit on its own
 * (the tensor-core path otherwise runs a k-wide conv and the 1x1 conv that
 * consumes only it as one launch, the intermediate kept on chip; the results
 * are identical). */
#define CC_FLAG_NO_UNIT_FUSION 1
/* cc_model_config.flags: launch sibling tensor-core convolutions on their own
 * (the path otherwise runs stride-1 convs that share their input, whose
 * outputs are read in FP32 only, as one contraction with their windows
 * right-aligned and their outputs side by side in one ring; the results are
 * identical). */
#define CC_FLAG_NO_SIBLING_MERGE 2

typedef struct cc_model cc_model;
typedef struct cc_stream cc_stream;

/* Build a model: validate the DAG, run the causal-reconfiguration analysis
 * (section 3: right pad -> left pad, Eq. 2 stride alignment, cumulated lag,
 * Eq. 3 branch alignment), size every cache, allocate the arena
 * (max_streams slots) and upload packed weights.
 * weights[i] / biases[i]: host float32 arrays for node i (NULL where the node
 * has none): conv [c_out][c_in][kernel], convt [c_in][c_out][kernel],
 * bias [c_out].  They are copied; the caller may free them on return.
 * Errors: INVALID_ARG, BAD_GRAPH (with the offending node in cc_last_error),
 * NO_MEMORY (also for an arena of 64 GiB or more: max_streams x slot size), CUDA. */
cc_status cc_model_create(const cc_node_desc* nodes, int32_t n_nodes,
                          const float* const* weights, const float* const* biases,
                          const cc_model_config* config, cc_model** out);
/* Frees the model, its arena and every stream still created on it (their
 * handles become invalid). */
cc_status cc_model_destroy(cc_model* model);

/* Total latency of the reconfigured model, in output frames: the cumulated
 * delay of the last node (section 3.1, section 4.3). */
cc_status cc_model_total_delay(const cc_model* model, int64_t* out_frames);

/* Channels and frames per model step.  A step is the smallest input length
 * that gives every layer a whole number of frames (e.g. 1 latent frame for a
 * x2048 decoder, 2048 samples for a /2048 encoder): the buffer granularity at
 * which strided layers stay aligned (section 3.1). */
cc_status cc_model_io(const cc_model* model, int32_t* in_channels, int32_t* out_channels,
                      int32_t* in_per_step, int32_t* out_per_step);

/* Per-node analysis results: cumulated delay D (own frames), Eq. 2 extra delay
 * D_a (strided convs), Eq. 3 alignment A_i of each input (merges), frames of
 * this node's output kept between calls (the cached padding of its consumers),
 * and the node's frames per model step.  Any output pointer may be NULL. */
cc_status cc_model_node_info(const cc_model* model, int32_t node, int64_t* delay,
                             int32_t* extra_delay, int32_t* align3, int32_t* kept_frames,
                             int32_t* frames_per_step);

/* Stream slots of the arena (its admission capacity) and how many are free. */
cc_status cc_model_capacity(const cc_model* model, int32_t* max_streams, int32_t* free_slots);

/* Bytes of persistent cache state per stream (the cached padding of section
 * 2.2; section 4.1 measures it as the streaming method's only extra memory),
 * and bytes of one arena slot (state plus per-call rows). */
cc_status cc_model_state_bytes(const cc_model* model, size_t* state_bytes, size_t* slot_bytes);

/* Create a stream: take a free arena slot (NO_MEMORY when none is left: admission
 * by cache memory), zero its caches -- the zero left padding of the causal
 * model (section 3) -- and wait for cuda_stream.  `seed` keys the heads' noise.
 * Destroy returns the slot (it synchronises the device first). */
cc_status cc_stream_create(cc_model* model, uint64_t seed, void* cuda_stream, cc_stream** out);
cc_status cc_stream_destroy(cc_stream* stream);

/* Zero the stream's caches and its step counter and restore the identity
 * input manipulation (below); waits for cuda_stream. */
cc_status cc_stream_reset(cc_stream* stream, void* cuda_stream);

/* Latent manipulation (section 5.1, Fig. 7; section 5.2): from the stream's
 * next model step on, every input frame x (input frame index t, counted from
 * the stream's start) enters the model as
 *   x'[c] = scale[c] * x[c] + bias[c] + noise[c] * u(t, c)
 * inside the kernel that writes the input into the stream's caches (two FP32
 * fused multiply-adds).  For a decoder the input is the latent: bias[c]
 * shifts dimension c, scale[c] = 0 with bias[c] = v replaces it by v, and
 * noise[c] adds uniform noise of that amplitude.  u(t, c) in [-1, 1) is the
 * SplitMix64 draw with counter t * channels + c from the generator seeded
 * with (stream seed XOR 0x6C6174656E742D6E), the same counter-based draw as
 * the heads' noise in a separate seed domain, so streamed and offline runs
 * see the same noise.  scale, bias and noise are host arrays of `channels`
 * floats (must equal the model's input channels; NULL means all 1 / 0 / 0;
 * values must be finite, else CC_ERR_INVALID_ARG).  They are copied to the
 * stream's slot with an asynchronous copy on cuda_stream, and the call
 * returns once the copy has completed: steps enqueued on cuda_stream after
 * the call, or on any stream after it returns, see the new values.  (With a
 * cc_server, call it while the stream has no request outstanding.)  A stream
 * starts with the identity (1, 0, 0) and cc_stream_reset restores it;
 * cc_stream_get_state does not carry it.  The hand-written backward does not
 * differentiate through a manipulation: cc_backward_begin and
 * cc_backward_chunk return CC_ERR_STATE for a stream that has one. */
cc_status cc_stream_set_input_manipulation(cc_stream* stream, const float* scale, const float* bias,
                                           const float* noise, int32_t channels, void* cuda_stream);

/* Process one buffer (cached padding, section 2.2 and Fig. 1: every layer
 * reads its last frames from the stream's caches in place of zero padding):
 * n_in input frames ([n_in][in_channels]) -> n_out output frames
 * ([n_out][out_channels]).  Outside FIFO mode n_in must be a multiple of
 * in_per_step and n_out == n_in / in_per_step * out_per_step (else
 * BAD_LENGTH).  The output of a call is the reconfigured model's output for
 * these frames: it equals the offline model's output delayed by
 * cc_model_total_delay frames (section 4.2).  In FIFO mode (below) any
 * lengths are accepted as long as the output asked for is queued or due. */
cc_status cc_stream_process(cc_stream* stream, const float* in, int64_t n_in, float* out,
                            int64_t n_out, void* cuda_stream);

/* Buffers that are not whole model steps (the paper's DSP call takes whatever
 * buffer the host hands it, section 1; its model steps are the strided
 * layers' alignment unit, section 3.1).  enable = 1 switches the stream to
 * FIFO mode: input frames short of a whole step wait in the stream's input
 * queue, a step runs as soon as its input is complete, and output frames wait
 * in an output queue until a call asks for them.  The output queue starts
 * with `prefill_frames` zero frames: the extra latency the caller accepts,
 * added to the stream's delay (cc_stream_delay).  A call may ask for at most
 * the queued frames plus those its input completes (else BAD_LENGTH, with no
 * state changed).  For fixed calls of b input and b' output frames, prefill =
 * out_per_step - gcd(b', out_per_step) serves every call (out_per_step - b'
 * when b' divides out_per_step); a caller that attaches each model step's input
 * to the first call needing its output needs none.  enable = 0 drops the
 * queues and returns to whole-step calls.  cc_stream_reset empties the input
 * queue and restores the prefill; the state blob does not carry the queues.
 * All calls of a FIFO-mode stream must be ordered on one CUDA stream.
 * Synchronises cuda_stream. */
cc_status cc_stream_set_fifo(cc_stream* stream, int32_t enable, int64_t prefill_frames, void* cuda_stream);
/* Latency of this stream's output, in output frames: cc_model_total_delay
 * plus the FIFO prefill (section 4.2's latency compensation). */
cc_status cc_stream_delay(const cc_stream* stream, int64_t* out_frames);
/* Frames waiting in the FIFO queues (0 outside FIFO mode); either pointer may be NULL. */
cc_status cc_stream_fifo_state(const cc_stream* stream, int64_t* in_frames, int64_t* out_frames);

/* Process one buffer for each of `count` distinct streams of one model
 * (a ragged batch): stream i gives n_in[i] input frames at in[i] and receives
 * n_out[i] output frames at out[i] (host or device pointers; in[i] / out[i]
 * may be NULL where the length is 0), each under cc_stream_process's length
 * rules for its mode.  Streams that run the same number of model steps share
 * one launch chain (streams batched into the contraction's N dimension); the
 * buffers are staged through device memory.  A stream may appear only once. */
cc_status cc_process_batch(cc_model* model, cc_stream* const* streams, const float* const* in,
                           const int64_t* n_in, float* const* out, const int64_t* n_out, int32_t count,
                           void* cuda_stream);

/* The fast form of cc_process_batch for equal-length buffers laid out with a
 * fixed stride (with device buffers there is no staging, so the call can be
 * captured in a CUDA graph):
 * in:  count buffers of n_in frames, stream i at in + i*in_stride (floats);
 * out: count buffers of n_out frames, stream i at out + i*out_stride.
 * Whole-step lengths only (cc_stream_process outside FIFO mode); streams in
 * FIFO mode are refused (STATE).  With host buffers in and out, the buffers go
 * through device staging of the CUDA stream's own, and the launch chain
 * between the copies is captured into a CUDA graph on its first use for that
 * number of streams and steps and replayed after (the first such call takes
 * the capture's time; a later autotuning, or staging that has to grow,
 * captures again). */
cc_status cc_process_batch_strided(cc_model* model, cc_stream* const* streams, int32_t count,
                                   const float* in, int64_t in_stride, int64_t n_in, float* out,
                                   int64_t out_stride, int64_t n_out, void* cuda_stream);

/* Checkpoint / resume (the paper has no counterpart): the whole stream state
 * (its arena slot, holding every cache of section 2.2, plus its step counter)
 * as an opaque host blob of exactly cc_stream_state_size() bytes.  Both calls
 * synchronise cuda_stream.  A blob restores into any stream of the same
 * model. */
cc_status cc_stream_state_size(const cc_stream* stream, size_t* bytes);
cc_status cc_stream_get_state(cc_stream* stream, void* host_blob, size_t bytes, void* cuda_stream);
cc_status cc_stream_set_state(cc_stream* stream, const void* host_blob, size_t bytes,
                              void* cuda_stream);

/* Failure detection (the paper has no counterpart).  Synchronises the device
 * and reports whether any tensor-core pipeline wait of this model gave up
 * since the last call (TIMEOUT, *code = bit set of the
 * waiting roles: 1 producer, 2 epilogue, 4 MMA issuer); clears the record.
 * Such a wait is bounded (cc_model_config.wait_limit_ns) so that a stalled
 * pipeline returns instead of hanging the GPU: the kernel lets the copies it
 * issued land, frees its tensor memory and exits; the affected outputs are
 * then undefined, and the streams of that call should be reset. */
cc_status cc_model_device_status(cc_model* model, int32_t* code);
/* Failure-detection test hook: each of the next `launches` tensor-core
 * launches of this model leaves, in its first CTA, the window rows of the
 * first K slice unrequested, so that CTA's pipeline waits run out after
 * wait_limit_ns and cc_model_device_status reports TIMEOUT.  Nothing faults
 * or hangs: every wait gives up and the kernel returns.  0 turns it off.
 * Synchronises the device.  STATE for a plan-only model. */
cc_status cc_model_test_withhold_copy(cc_model* model, int32_t launches);

/* Per-node device timing for measurement (the paper has no counterpart; its
 * section 4.1 times whole buffers).  CUDA events are recorded around every
 * launch on the launching stream.  enable=1 starts accumulating; cc_model_timing_read
 * synchronises and returns, per node, the summed milliseconds and launch count
 * since the last enable. */
cc_status cc_model_timing(cc_model* model, int32_t enable);
/* Kernels enqueued by the most recent launch chain of this model (one chain
 * covers up to max_steps_per_call steps of one batch): for launch accounting. */
cc_status cc_model_chain_launches(const cc_model* model, int32_t* launches);
cc_status cc_model_timing_read(cc_model* model, double* ms_per_node, int64_t* launches_per_node,
                               int32_t n_nodes);

/* ---------------------------------------------------------------- backward
 * Gradients of a loss over a long streamed signal, chunk by chunk in reverse
 * time order with per-chunk activation checkpointing.  The streamed output
 * equals the causal offline model (section 4.2), so these are that model's
 * gradients with respect to the input and to every weight and bias.  (The
 * paper trains offline and streams only at inference, section 4.3; this
 * chunked form has no counterpart there.)
 *
 * Protocol, for streams processed forward chunk by chunk:
 *   forward:  before chunk c, cc_snapshot_batch the streams into a device
 *             buffer (cc_model_snapshot_bytes per stream); process the chunk.
 *   backward: cc_backward_begin once; then for c = last .. first:
 *             cc_restore_batch the chunk-c snapshots and call
 *             cc_backward_chunk with chunk c's input and output gradient.
 * cc_backward_chunk recomputes the chunk's forward (the rings then hold its
 * activations), clears the adjoint rows no later chunk could have reached,
 * and propagates adjoints through the nodes in reverse order; the adjoint of
 * the cached frames a chunk read stays in the adjoint arena for the previous
 * chunk.  Weight / bias gradients accumulate in the cc_grads buffers.
 * FP32 models, and low-precision models created with CC_FLAG_NO_UNIT_FUSION
 * (STATE otherwise): the forward then runs in BF16/FP16 on the tensor cores
 * and the gradients are those of that arithmetic, in FP32 -- the backward
 * multiplies the rounded weights and the rounded activations the forward
 * multiplied (a rounding's derivative taken as 1).  All signal pointers are device memory:
 * x [n_in][in_channels], grad_y [n_out][out_channels], grad_x (may be NULL)
 * [n_in][in_channels], stream i at base + i*stride.  n_in is a whole number
 * of model steps, at most max_steps_per_call.  With grad_x NULL the adjoint
 * of the model input is not computed at all (weights only): pass grad_x for
 * every chunk of a backward pass or for none, since a chunk's input adjoint
 * includes what the later chunks carried back. */
typedef struct cc_grads cc_grads;
/* weights: the trained-layout float32 host weights the model was created with. */
cc_status cc_grads_create(cc_model* model, const float* const* weights, cc_grads** out);
cc_status cc_grads_destroy(cc_grads* grads);
cc_status cc_grads_zero(cc_grads* grads);
/* Host copies of one node's accumulated gradients (trained layouts); db may be NULL. */
cc_status cc_grads_read(cc_grads* grads, int32_t node, float* dw, float* db);
cc_status cc_backward_begin(cc_grads* grads, cc_stream* const* streams, int32_t count, void* cuda_stream);
cc_status cc_backward_chunk(cc_grads* grads, cc_stream* const* streams, int32_t count, const float* x,
                            int64_t x_stride, int64_t n_in, const float* grad_y, int64_t gy_stride,
                            int64_t n_out, float* grad_x, int64_t gx_stride, void* cuda_stream);

/* Device time of the backward's kernels by class, for measurement (no
 * counterpart in the paper): with timing enabled every kernel of
 * cc_backward_chunk is bracketed by CUDA events on the launching stream (it
 * adds a few microseconds per launch; keep it off when timing the whole pass).
 * cc_grads_timing(enable) synchronizes the device and clears what was
 * recorded; cc_grads_timing_read waits for the recorded kernels and returns,
 * per class, the summed milliseconds and the number of launches (arrays of
 * CC_BWD_CLASSES entries; either may be NULL). */
enum {
  CC_BWD_RECOMPUTE = 0, /* the chunk's forward, recomputed from the restored state */
  CC_BWD_CLEAR = 1,     /* zeroing adjoint rows no later chunk wrote (one launch)  */
  CC_BWD_DATA = 2,      /* dL/dx of a convolution (history rows included)          */
  CC_BWD_WEIGHT = 3,    /* dL/dW and dL/db of a convolution                        */
  CC_BWD_MERGE = 4,     /* residual adds and the heads                             */
  CC_BWD_INPUT = 5,     /* copy of the input adjoint out to grad_x                 */
  CC_BWD_CLASSES = 6
};
cc_status cc_grads_timing(cc_grads* grads, int32_t enable);
cc_status cc_grads_timing_read(cc_grads* grads, double* ms, int64_t* launches, int32_t n_classes);
/* The same per node: ms and launches are [n_nodes][CC_BWD_CLASSES] (the
 * recompute and the clear, which span every node, are left out). */
cc_status cc_grads_timing_read_nodes(cc_grads* grads, int32_t n_nodes, double* ms, int64_t* launches);

/* Device-side copies of streams' state for per-chunk checkpoints: the step
 * counter, the noise seed and the cached padding itself -- every ring's kept
 * rows (section 2.2's cache; section 4.1 measures it as the method's only
 * extra memory), not the whole arena slot.  cc_model_snapshot_bytes gives the
 * bytes per stream (16 + the cached state).  The batch forms copy `count`
 * distinct streams of one model, stream i at dev_buf + i * that size (bytes =
 * count x that size, dev_buf 8-byte aligned), with one kernel; restoring also
 * rewrites the mirrored rows of low-precision views.  Asynchronous on
 * cuda_stream. */
cc_status cc_model_snapshot_bytes(const cc_model* model, size_t* bytes);
cc_status cc_snapshot_batch(cc_model* model, cc_stream* const* streams, int32_t count, void* dev_buf, size_t bytes,
                            void* cuda_stream);
cc_status cc_restore_batch(cc_model* model, cc_stream* const* streams, int32_t count, const void* dev_buf,
                           size_t bytes, void* cuda_stream);
cc_status cc_stream_snapshot(cc_stream* stream, void* dev_buf, size_t bytes, void* cuda_stream);
cc_status cc_stream_restore(cc_stream* stream, const void* dev_buf, size_t bytes, void* cuda_stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of many real-time streams of one model: the paper's
 * per-buffer real-time processing (section 1, section 4.1) for many streams at
 * once; the paper itself runs one stream and has no server.  Clients submit
 * requests from any thread; a scheduler thread repeatedly advances, by one
 * model step and in one batched launch chain, every stream that has a request
 * still owed output and a full step of input buffered (oldest request first,
 * at most max_batch streams).  Streams that arrive while a batch is on the GPU
 * join the next batch; caches stay resident in the arena slots.  Output
 * beyond what a request asked for waits in the stream's FIFO, so requests
 * shorter than a model step are served from it.  Batch sizes are padded to a
 * multiple of `bucket` with a scratch stream slot (taken at creation); the
 * launch chain of each bucket is replayed from a CUDA graph (use_graphs) and
 * its tile shapes come from the model's autotuner (autotune: each
 * tensor-core layer is timed with 128- and 256-column tiles on the scratch
 * slot, three rounds alternating the two, and the smaller minimum is kept). */
typedef struct cc_server cc_server;
typedef struct {
  int32_t max_batch;  /* streams per launch chain, <= the model's max_streams - 1 */
  int32_t bucket;     /* batch sizes are padded to a multiple of this (0: 32)      */
  int32_t use_graphs; /* replay each bucket's launch chain from a CUDA graph        */
  int32_t autotune;   /* choose tensor-core tile shapes per bucket by timing         */
} cc_server_config;

/* Needs one free stream slot (the padding scratch); NO_MEMORY otherwise. */
cc_status cc_server_create(cc_model* model, const cc_server_config* config, cc_server** out);
/* Stops the scheduler after its current batch; pending requests are dropped. */
cc_status cc_server_destroy(cc_server* server);
/* count requests: request i gives stream streams[i] n_in[i] input frames
 * (host, [n_in][in_channels], copied in) and asks for n_out[i] output frames
 * written to the host buffer out[i] ([n_out][out_channels], written by the
 * scheduler thread; valid once cc_server_poll reports tags[i]).  A stream's
 * requests complete in order. */
cc_status cc_server_submit(cc_server* server, int32_t count, cc_stream* const* streams,
                           const float* const* in, const int64_t* n_in, float* const* out,
                           const int64_t* n_out, const uint64_t* tags);
/* Up to max completed requests: tag, submit time, start of the GPU step that
 * completed the request (its submit time when the stream's FIFO already held
 * the output) and completion time (ns, steady clock; every array may be
 * NULL).  Returns the scheduler's error if it stopped on one. */
cc_status cc_server_poll(cc_server* server, int32_t max, uint64_t* tags, int64_t* submit_ns,
                         int64_t* step_ns, int64_t* done_ns, int32_t* got);
/* Forgets a stream (its pending requests are dropped) once it is not in the
 * batch on the GPU; call before cc_stream_destroy of a served stream. */
cc_status cc_server_remove(cc_server* server, cc_stream* stream);
/* Batches run, stream-steps, time in GPU steps (ns), the largest batch, and
 * the first batches of a bucket (tuning, warm-up and graph capture: their
 * number and time, cc_server_prepare's included); any may be NULL. */
cc_status cc_server_stats(cc_server* server, int64_t* batches, int64_t* stream_steps,
                          int64_t* gpu_ns, int64_t* max_batch, int64_t* setups, int64_t* setup_ns);
/* Tunes, warms up and captures every bucket of batches up to max_count
 * streams now, so that no request later waits behind that set-up (it takes a
 * few milliseconds per bucket).  Waits for the batch on the GPU, holds the
 * scheduler off meanwhile; requests submitted during the call wait for it. */
cc_status cc_server_prepare(cc_server* server, int32_t max_count);

/* Host utility: a cosine-modulated pseudo-QMF bank (bands x taps) with a
 * Kaiser(beta) prototype whose cutoff minimises the prototype autocorrelation
 * at lags 2*bands*l (Lin & Vaidyanathan 1998).  analysis / synthesis:
 * [bands][taps] float64 (may be NULL); cutoff in rad/sample (may be NULL).
 * The paper uses such a bank inside RAVE (section 2.3) but does not specify it. */
cc_status cc_pqmf_design(int32_t bands, int32_t taps, double beta, double* analysis,
                         double* synthesis, double* cutoff);
/* The same bank as the trained-layout weights of the two PQMF layers of a
 * RAVE-like model: the analysis Conv1d(1 -> bands, kernel taps, stride bands),
 * [bands][1][taps] = g_b (correlating with g_b filters by its time reverse,
 * the analysis filter h_b), and the synthesis ConvTranspose1d(bands -> 1,
 * kernel taps, stride bands), [bands][1][taps] = bands * g_b (the factor M of
 * the cosine-modulated bank's reconstruction).  Either pointer may be NULL. */
cc_status cc_pqmf_layer_weights(int32_t bands, int32_t taps, double beta, float* analysis_conv,
                                float* synthesis_convt);

/* One cached Conv1d step that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * when they process a buffer, such as a real-time audio callback (cudaMalloc
 * may synchronise the device and take an unbounded time, heard as a dropout)
 * or a plug-in living inside a fixed, pre-reserved memory budget.
 *
 * Computes the same layer as a model [input, conv] through cc_stream_process:
 * y[t] = bias + sum_k W[:, :, k] . act(z[t + k*dilation]), where z is the
 * cached frames followed by x.  All device pointers, caller-owned:
 *   x      [n][c_in] input frames; y [n][c_out] output frames
 *   weight [c_out][c_in][kernel]; bias [c_out] or NULL
 *   cache  [pad_left + pad_right][c_in], oldest frame first: in/out, the
 *          frames kept between calls; all zero at the start of a stream
 * Scratch (packed weights and the window) lives in a 16 MiB device array
 * that every GPU loading this library holds until the process exits; a layer
 * needing more is rejected with CC_ERR_INVALID_ARG (message in
 * cc_last_error).  The call makes no cudaMalloc / cudaFree or other
 * allocating call.  Its first call on a device looks up that device's copy
 * of the array (with the device current); with the CUDA runtime's default
 * lazy module loading that first lookup also loads the library's device code
 * and reserves the array, which may allocate and synchronise.  So make one
 * warm-up call per device outside the real-time path and before any stream
 * capture: a call with n == 0 (the other pointers may then be NULL) does
 * exactly this set-up and nothing else.  All calls share the one array and
 * each overwrites it: calls that overlap on the GPU (different CUDA streams,
 * or other threads) race; serialise them on one stream.  No pointer needs
 * more than 4-byte alignment (the bias is copied into the array).
 * Asynchronous on cuda_stream. */
cc_status cc_cached_conv1d_static(const float* x, int64_t n, int32_t c_in, int32_t c_out,
                                  int32_t kernel, int32_t dilation, int32_t pad_left,
                                  int32_t pad_right, int32_t act_in, const float* weight,
                                  const float* bias, float* cache, float* y, void* cuda_stream);

const char* cc_status_str(cc_status status);
const char* cc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CACHEDCONV_H */
