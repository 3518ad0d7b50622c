"""Thin Python binding of ``include/cachedconv.h`` (argument marshalling only).

Every step of the streamed model runs in the CUDA library; this module only
converts node dictionaries and weights to the C structures and passes
pointers.  Device buffers are torch CUDA tensors (float32, contiguous); host
buffers are numpy float32 arrays or CPU tensors (staged by the library).
If the compiled library is missing, every entry point raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

OPS = {"input": 0, "conv": 1, "convt": 2, "add": 3, "heads": 4}
ACTS = {None: 0, "leaky": 1}
DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
STATUS = {0: "ok", -1: "invalid argument", -2: "bad graph", -3: "bad length",
          -4: "no memory", -5: "cuda error", -6: "timeout", -7: "bad state"}


class CCError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class NodeDesc(C.Structure):
    _fields_ = [("op", C.c_int32), ("n_inputs", C.c_int32), ("inputs", C.c_int32 * 3),
                ("c_in", C.c_int32), ("c_out", C.c_int32), ("kernel", C.c_int32),
                ("stride", C.c_int32), ("dilation", C.c_int32), ("pad_left", C.c_int32),
                ("pad_right", C.c_int32), ("crop", C.c_int32), ("act_in", C.c_int32),
                ("has_bias", C.c_int32)]


class ModelConfig(C.Structure):
    _fields_ = [("compute", C.c_int32), ("max_streams", C.c_int32),
                ("max_steps_per_call", C.c_int32), ("noise", C.c_int32), ("flags", C.c_int32),
                ("arena_bytes", C.c_int64), ("wait_limit_ns", C.c_int64)]


_LIB = None
_P = C.c_void_p
_I32, _I64, _U64, _SZ, _DBL = C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_double

_SIGNATURES = {
    "cc_model_create": [C.POINTER(NodeDesc), _I32, C.POINTER(_P), C.POINTER(_P),
                        C.POINTER(ModelConfig), C.POINTER(_P)],
    "cc_model_destroy": [_P],
    "cc_model_total_delay": [_P, C.POINTER(_I64)],
    "cc_model_io": [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)],
    "cc_model_node_info": [_P, _I32, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I32),
                           C.POINTER(_I32), C.POINTER(_I32)],
    "cc_model_state_bytes": [_P, C.POINTER(_SZ), C.POINTER(_SZ)],
    "cc_stream_create": [_P, _U64, _P, C.POINTER(_P)],
    "cc_stream_destroy": [_P],
    "cc_stream_reset": [_P, _P],
    "cc_stream_set_input_manipulation": [_P, _P, _P, _P, _I32, _P],
    "cc_stream_process": [_P, _P, _I64, _P, _I64, _P],
    "cc_model_capacity": [_P, C.POINTER(_I32), C.POINTER(_I32)],
    "cc_stream_set_fifo": [_P, _I32, _I64, _P],
    "cc_stream_delay": [_P, C.POINTER(_I64)],
    "cc_stream_fifo_state": [_P, C.POINTER(_I64), C.POINTER(_I64)],
    "cc_process_batch": [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_I64), C.POINTER(_P), C.POINTER(_I64),
                         _I32, _P],
    "cc_process_batch_strided": [_P, C.POINTER(_P), _I32, _P, _I64, _I64, _P, _I64, _I64, _P],
    "cc_stream_state_size": [_P, C.POINTER(_SZ)],
    "cc_stream_get_state": [_P, _P, _SZ, _P],
    "cc_stream_set_state": [_P, _P, _SZ, _P],
    "cc_model_device_status": [_P, C.POINTER(_I32)],
    "cc_model_test_withhold_copy": [_P, _I32],
    "cc_model_timing": [_P, _I32],
    "cc_model_chain_launches": [_P, C.POINTER(_I32)],
    "cc_model_timing_read": [_P, C.POINTER(_DBL), C.POINTER(_I64), _I32],
    "cc_pqmf_design": [_I32, _I32, _DBL, C.POINTER(_DBL), C.POINTER(_DBL), C.POINTER(_DBL)],
    "cc_pqmf_layer_weights": [_I32, _I32, _DBL, _P, _P],
    "cc_cached_conv1d_static": [_P, _I64, _I32, _I32, _I32, _I32, _I32, _I32, _I32, _P, _P, _P,
                                _P, _P],
    "cc_server_create": [_P, C.c_void_p, C.POINTER(_P)],
    "cc_server_destroy": [_P],
    "cc_server_submit": [_P, _I32, _P, _P, _P, _P, _P, _P],
    "cc_server_poll": [_P, _I32, _P, _P, _P, _P, C.POINTER(_I32)],
    "cc_server_prepare": [_P, _I32],
    "cc_server_remove": [_P, _P],
    "cc_server_stats": [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64),
                        C.POINTER(_I64)],
    "cc_grads_create": [_P, C.POINTER(_P), C.POINTER(_P)],
    "cc_grads_destroy": [_P],
    "cc_grads_zero": [_P],
    "cc_grads_read": [_P, _I32, _P, _P],
    "cc_backward_begin": [_P, _P, _I32, _P],
    "cc_backward_chunk": [_P, _P, _I32, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, _P],
    "cc_grads_timing": [_P, _I32],
    "cc_grads_timing_read": [_P, C.POINTER(_DBL), C.POINTER(_I64), _I32],
    "cc_grads_timing_read_nodes": [_P, _I32, C.POINTER(_DBL), C.POINTER(_I64)],
    "cc_model_snapshot_bytes": [_P, C.POINTER(_SZ)],
    "cc_snapshot_batch": [_P, C.POINTER(_P), _I32, _P, _SZ, _P],
    "cc_restore_batch": [_P, C.POINTER(_P), _I32, _P, _SZ, _P],
    "cc_stream_snapshot": [_P, _P, _SZ, _P],
    "cc_stream_restore": [_P, _P, _SZ, _P],
    "cc_status_str": [_I32],
    "cc_last_error": [],
}

EXPORTED = tuple(_SIGNATURES)


def library_path():
    return _build.LIB


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name in ("cc_status_str", "cc_last_error") else C.c_int32
        _LIB = L
    return _LIB


def _check(status):
    if status != 0:
        raise CCError(status, lib().cc_last_error().decode())


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (float32, contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float32 and x.flags.c_contiguous
        return x.ctypes.data
    assert x.dtype.__str__().endswith("float32") and x.is_contiguous()
    return x.data_ptr()


def _cuda_stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _desc(node):
    d = NodeDesc()
    d.op = OPS[node["op"]]
    ins = list(node["inputs"])
    d.n_inputs = len(ins)
    for i, v in enumerate(ins):
        d.inputs[i] = v
    d.c_in, d.c_out = node["c_in"], node["c_out"]
    d.kernel, d.stride, d.dilation = node["k"], node["stride"], node["dilation"]
    d.pad_left, d.pad_right, d.crop = node["pad_left"], node["pad_right"], node["crop"]
    d.act_in = ACTS[node["act_in"]]
    d.has_bias = int(bool(node["bias"]))
    return d


class Model:
    """A reconfigured model on the GPU: packed weights + stream-state arena.

    dtype "f32" runs FFMA kernels; "bf16" / "f16" run the contractions with
    cin % 64 == 0 and cout % 8 == 0 on the tensor cores.  max_streams sizes the arena (0: plan
    only); max_steps_per_call is the longest launch chain (longer buffers are
    split).  fuse_units / merge_siblings = False launch each convolution of a
    residual unit, and each sibling conv, on its own (identical results; for
    comparisons).  arena_bytes > 0 sizes the arena by bytes (admission by
    cache memory); wait_limit_ns bounds every device-side pipeline wait."""

    def __init__(self, nodes, params, dtype="f32", max_streams=1, max_steps_per_call=1, noise=True,
                 fuse_units=True, merge_siblings=True, arena_bytes=0, wait_limit_ns=0):
        L = lib()
        n = len(nodes)
        descs = (NodeDesc * n)(*[_desc(nd) for nd in nodes])
        self._keep = []
        wp = (_P * n)()
        bp = (_P * n)()
        for i, nd in enumerate(nodes):
            if i in params:
                w, b = params[i]
                w32 = np.ascontiguousarray(w, dtype=np.float32)
                self._keep.append(w32)
                wp[i] = w32.ctypes.data
                if b is not None:
                    b32 = np.ascontiguousarray(b, dtype=np.float32)
                    self._keep.append(b32)
                    bp[i] = b32.ctypes.data
        cfg = ModelConfig(DTYPES[dtype], max_streams, max_steps_per_call, int(bool(noise)),
                          (0 if fuse_units else 1) | (0 if merge_siblings else 2), int(arena_bytes),
                          int(wait_limit_ns))
        h = _P()
        _check(L.cc_model_create(descs, n, wp, bp, C.byref(cfg), C.byref(h)))
        self._keep = None
        self._streams = weakref.WeakSet()
        self.handle = h
        self.nodes = nodes
        self.dtype = dtype
        self.max_steps_per_call = max_steps_per_call
        self.max_streams = self.capacity[0] if (max_streams or arena_bytes) else 0

    def close(self):
        if getattr(self, "handle", None):
            for s in list(self._streams):  # the library frees them with the model
                s.handle = None
            _check(lib().cc_model_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def total_delay(self):
        v = _I64()
        _check(lib().cc_model_total_delay(self.handle, C.byref(v)))
        return v.value

    @property
    def io(self):
        a, b, c, d = _I32(), _I32(), _I32(), _I32()
        _check(lib().cc_model_io(self.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return dict(in_channels=a.value, out_channels=b.value, in_per_step=c.value,
                    out_per_step=d.value)

    def node_info(self, i):
        d, da, k, u = _I64(), _I32(), _I32(), _I32()
        al = (_I32 * 3)()
        _check(lib().cc_model_node_info(self.handle, i, C.byref(d), C.byref(da), al, C.byref(k), C.byref(u)))
        return dict(delay=d.value, extra_delay=da.value, align=list(al), kept=k.value,
                    frames_per_step=u.value)

    @property
    def capacity(self):
        """(stream slots of the arena, free slots)."""
        a, b = _I32(), _I32()
        _check(lib().cc_model_capacity(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    @property
    def state_bytes(self):
        a, b = _SZ(), _SZ()
        _check(lib().cc_model_state_bytes(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def stream(self, seed=0, cuda_stream=None):
        return Stream(self, seed, cuda_stream)

    def process_batch(self, streams, x, y, cuda_stream=None):
        """Equal-length buffers (cc_process_batch_strided): x [count][n_in][C_in],
        y [count][n_out][C_out] float32 (device or host)."""
        count = len(streams)
        arr = (_P * count)(*[s.handle for s in streams])
        n_in = x.shape[1]
        n_out = y.shape[1]
        in_stride = int(np.prod(x.shape[1:]))
        out_stride = int(np.prod(y.shape[1:]))
        _check(lib().cc_process_batch_strided(self.handle, arr, count, _ptr(x), in_stride, n_in, _ptr(y),
                                              out_stride, n_out, _cuda_stream(cuda_stream)))

    def process_ragged(self, streams, xs, ys, cuda_stream=None):
        """A ragged batch (cc_process_batch): stream i reads xs[i] [n_in_i][C_in]
        and writes ys[i] [n_out_i][C_out] (float32, device or host; None for
        an empty buffer)."""
        count = len(streams)
        arr = (_P * count)(*[s.handle for s in streams])
        ip = (_P * count)(*[None if x is None else _ptr(x) for x in xs])
        op = (_P * count)(*[None if y is None else _ptr(y) for y in ys])
        ni = (_I64 * count)(*[0 if x is None else x.shape[0] for x in xs])
        no = (_I64 * count)(*[0 if y is None else y.shape[0] for y in ys])
        _check(lib().cc_process_batch(self.handle, arr, ip, ni, op, no, count, _cuda_stream(cuda_stream)))

    def device_status(self):
        """Raises CCError(TIMEOUT) if a bounded device wait gave up since the last call."""
        code = _I32()
        _check(lib().cc_model_device_status(self.handle, C.byref(code)))
        return code.value

    def device_status_code(self):
        """(status, role bits) of cc_model_device_status, without raising."""
        code = _I32()
        st = lib().cc_model_device_status(self.handle, C.byref(code))
        return st, code.value

    def test_withhold_copy(self, launches=1):
        """Failure-detection test hook (cc_model_test_withhold_copy)."""
        _check(lib().cc_model_test_withhold_copy(self.handle, int(launches)))

    @property
    def chain_launches(self):
        """Kernels the most recent launch chain enqueued."""
        v = _I32()
        _check(lib().cc_model_chain_launches(self.handle, C.byref(v)))
        return v.value

    def timing(self, enable):
        _check(lib().cc_model_timing(self.handle, int(enable)))

    def timing_read(self):
        n = len(self.nodes)
        ms = (_DBL * n)()
        cnt = (_I64 * n)()
        _check(lib().cc_model_timing_read(self.handle, ms, cnt, n))
        return list(ms), list(cnt)


class Stream:
    """Per-stream cache state (one arena slot)."""

    def __init__(self, model, seed=0, cuda_stream=None):
        self.model = model
        h = _P()
        _check(lib().cc_stream_create(model.handle, seed & (2 ** 64 - 1),
                                      _cuda_stream(cuda_stream) if _has_cuda() else None, C.byref(h)))
        self.handle = h
        self.seed = seed
        model._streams.add(self)

    def process(self, x, y, cuda_stream=None):
        """x: [n_in][C_in], y: [n_out][C_out] float32 (device or host buffers)."""
        _check(lib().cc_stream_process(self.handle, _ptr(x), x.shape[0], _ptr(y), y.shape[0],
                                       _cuda_stream(cuda_stream)))

    def reset(self, cuda_stream=None):
        _check(lib().cc_stream_reset(self.handle, _cuda_stream(cuda_stream)))

    def set_fifo(self, enable=True, prefill=0, cuda_stream=None):
        """FIFO mode: buffers of any length; the output queue starts with
        `prefill` zero frames (added to the stream's delay)."""
        _check(lib().cc_stream_set_fifo(self.handle, int(bool(enable)), int(prefill), _cuda_stream(cuda_stream)))

    @property
    def delay(self):
        """Output latency of this stream in output frames (model delay + FIFO prefill)."""
        v = _I64()
        _check(lib().cc_stream_delay(self.handle, C.byref(v)))
        return v.value

    @property
    def fifo_state(self):
        a, b = _I64(), _I64()
        _check(lib().cc_stream_fifo_state(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_input_manipulation(self, scale=None, bias=None, noise=None, cuda_stream=None):
        """Latent manipulation: from the next step on, input frames enter the
        model as scale * x + bias + noise * u per channel, u a seeded uniform
        draw in [-1, 1) (None: 1 / 0 / 0; scalars broadcast).  Replace channel
        c by v with scale[c] = 0, bias[c] = v."""
        n = self.model.io["in_channels"]
        arrs = [None if v is None else np.ascontiguousarray(np.broadcast_to(v, (n,)), dtype=np.float32)
                for v in (scale, bias, noise)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        _check(lib().cc_stream_set_input_manipulation(self.handle, ptrs[0], ptrs[1], ptrs[2], n,
                                                      _cuda_stream(cuda_stream)))

    def get_state(self, cuda_stream=None):
        n = _SZ()
        _check(lib().cc_stream_state_size(self.handle, C.byref(n)))
        blob = np.empty(n.value, dtype=np.uint8)
        _check(lib().cc_stream_get_state(self.handle, blob.ctypes.data, n.value, _cuda_stream(cuda_stream)))
        return blob

    def set_state(self, blob, cuda_stream=None):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().cc_stream_set_state(self.handle, blob.ctypes.data, blob.size, _cuda_stream(cuda_stream)))

    def close(self):
        if getattr(self, "handle", None) and getattr(self.model, "handle", None):
            _check(lib().cc_stream_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _has_cuda():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def pqmf_design(bands=16, taps=64, beta=5.0):
    """Host PQMF design (analysis h, synthesis g as [bands][taps] float64, cutoff)."""
    h = np.zeros((bands, taps))
    g = np.zeros((bands, taps))
    wc = _DBL()
    _check(lib().cc_pqmf_design(bands, taps, beta, h.ctypes.data_as(C.POINTER(_DBL)),
                                g.ctypes.data_as(C.POINTER(_DBL)), C.byref(wc)))
    return h, g, wc.value


def pqmf_layer_weights(bands=16, taps=64, beta=5.0):
    """Trained-layout weights of the PQMF layers (cc_pqmf_layer_weights):
    analysis Conv(1 -> bands) [bands][1][taps] and synthesis
    ConvT(bands -> 1) [bands][1][taps], float32."""
    a = np.zeros((bands, 1, taps), np.float32)
    s = np.zeros((bands, 1, taps), np.float32)
    _check(lib().cc_pqmf_layer_weights(bands, taps, beta, a.ctypes.data, s.ctypes.data))
    return a, s


def cached_conv1d_static(x, weight, bias, cache, y, dilation=1, pad_left=0, pad_right=0,
                         act_in=None, cuda_stream=None):
    """One cached Conv1d step without any device allocation (see
    cc_cached_conv1d_static in include/cachedconv.h).  x [n][c_in],
    weight [c_out][c_in][K], bias [c_out] or None, cache [pad_left+pad_right][c_in]
    (updated in place), y [n][c_out]: float32 CUDA tensors."""
    n, c_in = x.shape
    c_out, _, k = weight.shape
    _check(lib().cc_cached_conv1d_static(
        _ptr(x), n, c_in, c_out, k, dilation, pad_left, pad_right, ACTS[act_in], _ptr(weight),
        None if bias is None else _ptr(bias), _ptr(cache) if cache.numel() else None, _ptr(y),
        _cuda_stream(cuda_stream)))


def cached_conv1d_static_warmup(cuda_stream=None):
    """The set-up of cc_cached_conv1d_static on the current device (an empty
    call): looks up the device's copy of the static scratch, which may load
    the library's device code.  Call once per device before the real-time
    path and before any stream capture."""
    _check(lib().cc_cached_conv1d_static(None, 0, 1, 1, 1, 1, 0, 0, 0, None, None, None, None,
                                         _cuda_stream(cuda_stream)))



class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("bucket", C.c_int32), ("use_graphs", C.c_int32),
                ("autotune", C.c_int32)]


class Server:
    """Continuous-batching scheduler of the library (cc_server_*): requests
    are host numpy buffers; completion times come back from poll()."""

    def __init__(self, model, max_batch, bucket=32, use_graphs=True, autotune=True):
        cfg = ServerConfig(max_batch, bucket, int(bool(use_graphs)), int(bool(autotune)))
        h = _P()
        _check(lib().cc_server_create(model.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self.model = model
        self._keep = []

    def submit(self, streams, ins, n_in, outs, n_out, tags):
        """streams: list of Stream; ins / outs: sequences of float32 numpy
        arrays (or raw addresses as uint64) -- the caller keeps them alive until
        completion; n_in / n_out: frames; tags: uint64."""
        count = len(streams)
        if count == 0:
            return
        sp = np.array([s.handle.value for s in streams], dtype=np.uint64)
        ip = np.asarray([x if isinstance(x, (int, np.integer)) else (0 if x is None else x.ctypes.data)
                         for x in ins], dtype=np.uint64)
        op = np.asarray([x if isinstance(x, (int, np.integer)) else (0 if x is None else x.ctypes.data)
                         for x in outs], dtype=np.uint64)
        ni = np.ascontiguousarray(n_in, dtype=np.int64)
        no = np.ascontiguousarray(n_out, dtype=np.int64)
        tg = np.ascontiguousarray(tags, dtype=np.uint64)
        _check(lib().cc_server_submit(self.handle, count, sp.ctypes.data, ip.ctypes.data, ni.ctypes.data,
                                      op.ctypes.data, no.ctypes.data, tg.ctypes.data))

    def submit_raw(self, count, stream_ptrs, in_ptrs, n_in, out_ptrs, n_out, tags):
        """Same as submit() with uint64 / int64 numpy arrays of addresses."""
        if count:
            _check(lib().cc_server_submit(self.handle, count, stream_ptrs.ctypes.data, in_ptrs.ctypes.data,
                                          n_in.ctypes.data, out_ptrs.ctypes.data, n_out.ctypes.data,
                                          tags.ctypes.data))

    def poll(self, max_items=65536, detail=False):
        """(tags, submit_ns, done_ns) of completed requests; with detail=True
        also the start of the GPU step that completed each (before done_ns)."""
        tags = np.empty(max_items, np.uint64)
        sub = np.empty(max_items, np.int64)
        step = np.empty(max_items, np.int64)
        done = np.empty(max_items, np.int64)
        got = _I32()
        _check(lib().cc_server_poll(self.handle, max_items, tags.ctypes.data, sub.ctypes.data, step.ctypes.data,
                                    done.ctypes.data, C.byref(got)))
        n = got.value
        if detail:
            return tags[:n], sub[:n], step[:n], done[:n]
        return tags[:n], sub[:n], done[:n]

    def prepare(self, max_count):
        """Tune and capture every batch bucket up to max_count streams now."""
        _check(lib().cc_server_prepare(self.handle, int(max_count)))

    def remove(self, stream):
        _check(lib().cc_server_remove(self.handle, stream.handle))

    def stats(self):
        v = [_I64() for _ in range(6)]
        _check(lib().cc_server_stats(self.handle, *[C.byref(x) for x in v]))
        return dict(batches=v[0].value, stream_steps=v[1].value, gpu_ns=v[2].value, max_batch=v[3].value,
                    setups=v[4].value, setup_ns=v[5].value)

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().cc_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



def snapshot_bytes(model):
    """Bytes of one stream's checkpoint: counter, seed and the cached state."""
    v = _SZ()
    _check(lib().cc_model_snapshot_bytes(model.handle, C.byref(v)))
    return v.value


def snapshot_batch(model, streams, buf, cuda_stream=None):
    """Checkpoints of `streams` into a uint8 CUDA tensor of len(streams) x snapshot_bytes."""
    arr = (_P * len(streams))(*[s.handle for s in streams])
    _check(lib().cc_snapshot_batch(model.handle, arr, len(streams), buf.data_ptr(), buf.numel(),
                                   _cuda_stream(cuda_stream)))


def restore_batch(model, streams, buf, cuda_stream=None):
    arr = (_P * len(streams))(*[s.handle for s in streams])
    _check(lib().cc_restore_batch(model.handle, arr, len(streams), buf.data_ptr(), buf.numel(),
                                  _cuda_stream(cuda_stream)))


class Grads:
    """Gradient accumulators + adjoint arena of a model (cc_grads_*): FP32, or
    low precision created with fuse_units=False."""

    def __init__(self, model, params):
        n = len(model.nodes)
        wp = (_P * n)()
        self._keep = []
        for i in range(n):
            if i in params:
                w32 = np.ascontiguousarray(params[i][0], dtype=np.float32)
                self._keep.append(w32)
                wp[i] = w32.ctypes.data
        h = _P()
        _check(lib().cc_grads_create(model.handle, wp, C.byref(h)))
        self._keep = None
        self.handle = h
        self.model = model

    def zero(self):
        _check(lib().cc_grads_zero(self.handle))

    def read(self, node):
        nd = self.model.nodes[node]
        from .workloads import weight_shape
        dw = np.zeros(weight_shape(nd), np.float32)
        db = np.zeros(nd["c_out"], np.float32) if nd["bias"] else None
        _check(lib().cc_grads_read(self.handle, node, dw.ctypes.data, None if db is None else db.ctypes.data))
        return dw, db

    def begin(self, streams, cuda_stream=None):
        arr = (_P * len(streams))(*[s.handle for s in streams])
        _check(lib().cc_backward_begin(self.handle, arr, len(streams), _cuda_stream(cuda_stream)))

    def chunk(self, streams, x, gy, gx=None, cuda_stream=None):
        """x [count][n_in][C_in], gy [count][n_out][C_out], gx like x (or None): CUDA tensors."""
        arr = (_P * len(streams))(*[s.handle for s in streams])
        _check(lib().cc_backward_chunk(self.handle, arr, len(streams), _ptr(x), int(np.prod(x.shape[1:])),
                                       x.shape[1], _ptr(gy), int(np.prod(gy.shape[1:])), gy.shape[1],
                                       None if gx is None else _ptr(gx),
                                       int(np.prod(x.shape[1:])), _cuda_stream(cuda_stream)))

    BWD_CLASSES = ("recompute", "clear", "data", "weight", "merge", "input")

    def timing(self, enable):
        """Bracket every backward kernel with CUDA events (cc_grads_timing)."""
        _check(lib().cc_grads_timing(self.handle, int(bool(enable))))

    def timing_read(self):
        """{class: (milliseconds, launches)} recorded since timing(True)."""
        n = len(self.BWD_CLASSES)
        ms, cnt = (_DBL * n)(), (_I64 * n)()
        _check(lib().cc_grads_timing_read(self.handle, ms, cnt, n))
        return {c: (ms[i], cnt[i]) for i, c in enumerate(self.BWD_CLASSES)}

    def timing_read_nodes(self):
        """[(node, class, milliseconds, launches)] with launches > 0."""
        n, k = len(self.model.nodes), len(self.BWD_CLASSES)
        ms, cnt = (_DBL * (n * k))(), (_I64 * (n * k))()
        _check(lib().cc_grads_timing_read_nodes(self.handle, n, ms, cnt))
        return [(i, c, ms[i * k + j], cnt[i * k + j]) for i in range(n) for j, c in enumerate(self.BWD_CLASSES)
                if cnt[i * k + j]]

    def close(self):
        if getattr(self, "handle", None) and getattr(self.model, "handle", None):
            _check(lib().cc_grads_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stream_snapshot(stream, buf, cuda_stream=None):
    """Device copy of a stream's state into a uint8 CUDA tensor of snapshot_bytes()."""
    _check(lib().cc_stream_snapshot(stream.handle, buf.data_ptr(), buf.numel(), _cuda_stream(cuda_stream)))


def stream_restore(stream, buf, cuda_stream=None):
    _check(lib().cc_stream_restore(stream.handle, buf.data_ptr(), buf.numel(), _cuda_stream(cuda_stream)))
