"""GB300-native streamed inference of non-causal 1-D convolutional audio models.

Post-training causal reconfiguration and cached padding (Caillon & Esling,
"Streamable neural audio synthesis with non-causal convolutions", DAFx-22),
as hand-written CUDA kernels for sm_103a behind a C ABI (``include/cachedconv.h``).
The Python side only marshals arguments; see ``paper_2204_07064_gb300.api``.
"""
