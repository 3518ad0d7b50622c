"""GB300-native streamed inference of non-causal 1-D convolutional audio models.

Post-training causal reconfiguration and cached padding (Caillon & Esling,
"Streamable neural audio synthesis with non-causal convolutions", DAFx-22),
as hand-written CUDA kernels for sm_103a behind a C ABI (``include/cachedconv.h``).
The Python side only marshals arguments:

* ``api.Model`` -- a layer list and trained weights; the causal
  reconfiguration (section 3), the stream arena and packed weights.
  ``api.Stream`` -- one audio stream's caches (section 2.2): ``process``,
  ``reset``, checkpoint / restore, ``set_input_manipulation`` (sections 5.1
  and 5.2).  ``Model.process_batch`` advances many streams in one launch chain.
* ``api.Server`` -- continuous batching of real-time streams.
* ``autograd.streamed`` -- the chunked backward behind ``torch.autograd``.
* ``workloads`` -- layer lists of the RAVE-like decoder and encoder (and their
  chain, audio -> audio) and seeded inputs.
* ``build.build()`` -- compiles the library in-tree with nvcc.
"""
