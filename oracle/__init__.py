"""FP64 CPU oracle for streamed non-causal convolutional audio models.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test suite, the smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library; it is a
plain, slow, obviously-correct restatement of the paper (Caillon & Esling,
"Streamable neural audio synthesis with non-causal convolutions", DAFx-22):

* ``conv``   Eq. 1 (1-D cross-correlation) with zero padding, stride and
             dilation (section 2.1); transposed convolution (section 2.1).
* ``model``  the post-training causal reconfiguration (section 3): right
             padding moved to the left, stride alignment (Eq. 2), cumulative
             lag (section 3.1), branch alignment (Eq. 3); the offline
             non-causal model, the offline causal model and an independent
             cached-padding streaming implementation (Fig. 1, section 2.2).
* ``pqmf``   the cosine-modulated pseudo-QMF bank of the RAVE-like model
             (Kaiser-window prototype).  The paper does not define it (parity
             of the design itself is checked by properties, not by the paper).
* ``noise``  SplitMix64 (Steele, Lea & Flood 2014) as a counter-based
             generator for the deterministic noise branch.
* ``metrics`` Eq. 4 / Eq. 5 distances and the SNR / max-abs checks.
* ``manipulate`` per-dimension scale, bias and noise of the model input
             (latent manipulation, sections 5.1 and 5.2).

All floating point is numpy float64.
"""
