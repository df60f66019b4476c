"""Plain FP64 CPU oracle for EDPC's online-learning compressor.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
run this package. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It restates the method of "EDPC: Accelerating Lossless Compression via
Lightweight Probability Models and Decoupled Parallel Dataflow"
(ACM MM 2025) step by step, in NumPy FP64:

* ``rng``      counter-based SplitMix64 used to draw the initial parameters.
* ``model``    the probability model: byte embedding, MBRB blocks (Sec. 3.1.2,
               Eqs. 9-13), LTE with the per-stream Feature Distribution
               Matrix (Sec. 3.2, Eqs. 14-16), 256-way head; its analytic
               adjoint; and Adam (Sec. 4.1).
* ``coder``    softmax-to-integer-CDF quantizer and a 32-bit range coder
               (the arithmetic coding of Sec. 2.1).
* ``compress`` Algorithm 1 run over b parallel streams (the batch of
               Sec. 3.3), for encoding and for decoding.

It shares no code with the CUDA path. Where the paper is silent, the
reading taken is stated in the docstring of the function that uses it.
Parity status of each function is stated in its module header.
"""
from .rng import splitmix64, init_values  # noqa: F401
from .model import Config, Model, param_layout  # noqa: F401
from .coder import quantize_cdf, RangeEncoder, RangeDecoder  # noqa: F401
from .compress import split_streams, oracle_compress, oracle_decompress  # noqa: F401
