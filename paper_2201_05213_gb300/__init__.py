"""GB300 (sm_103a) parallel decoding for a local autoregressive image compressor.

Implements the wavefront schedule of "Parallel Neural Local Lossless
Compression" (Algorithm 1, Section 3) and the adjacent-patch variant as
hand-written CUDA kernels behind the C ABI of include/nlc.h.  Submodules:

* ``nlc``    -- ctypes binding of the C ABI (same function names);
* ``codec``  -- buffer allocation / status checks on top of it;
* ``synth``  -- seeded synthetic images and initial weights;
* ``build``  -- nvcc build of libnlc.so.

Importing the package does not load the CUDA library; the first binding
call does, and fails loudly if it is missing.
"""

__all__ = ["nlc", "codec", "synth", "build"]
