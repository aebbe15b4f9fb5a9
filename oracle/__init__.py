"""FP64 CPU oracle for the streaming DeepClean -> whiten -> BBHnet path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  The CUDA library never imports, links or calls it, and it
shares no code, table or constant generator with the library: the two meet
only in the seeded inputs of ``paper_2108_12430_gb300.synth``.

Every function is a plain, slow, direct statement of what the method
computes, in float64, with NumPy matmuls as the only library primitive:

* ``layers``  - Conv1d, ConvTranspose1d, eval-mode BatchNorm, the BatchNorm
  fold, activations, global average pool, linear head.
* ``nets``    - DeepClean-shaped autoencoder and BBHnet-shaped classifier,
  layer by layer in the order the layer tables give.
* ``fir``     - FIR design from a PSD by a direct inverse DFT (whitening,
  anti-alias decimator, band-limited loss weight) and valid-mode filtering.
* ``stream``  - snapshot windows of a stream (Methods, "Streaming IaaS") and
  aggregation of overlapping predictions (Methods, "Data aggregation" and
  "Aggregation latency").
* ``grad``    - the band-limited PSD-weighted training loss and its exact
  reverse-mode gradient for DeepClean.
* ``quant``   - round-to-nearest-even casts to bfloat16 and float8 e4m3.

Readings of the paper where it is silent are listed in each module header;
the architecture itself is not in the paper (the paper only names the
models), so model-level fidelity to the paper's trained networks is
"parity unpinned": the oracle pins the *operations*, not the paper's weights.
"""
