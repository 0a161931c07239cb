"""Plain, slow, FP64 CPU oracle for the M-TIP slice / match / merge path.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU product path never imports, calls or links it, and this
package imports nothing from the product package.

What it computes (arXiv 2109.05339, Sec. II):

* ``nudft``     -- the direct non-uniform DFT sums, type 2 (slicing, Sec. II-A)
                   and type 1 (its adjoint, Sec. II-C), written as definitions.
* ``nufft``     -- a plain exponential-of-semicircle NUFFT (the FINUFFT method
                   the paper cites in Sec. II and III-A), step by step:
                   deconvolve, pad, FFT, interpolate -- and its exact transpose.
* ``rotation``  -- quaternion to rotation matrix and detector q-points to NUFFT
                   coordinates (the nonuniform points q_k of Table I).
* ``slicing``   -- model images as Re(type-2) at rotated detector points
                   (Sec. II-A), the adjoint, and the gradient of the slice loss.
* ``matching``  -- brute-force squared Euclidean distances, argmin with ties to
                   the lowest orientation index, top-k, best/second-best margin
                   (Sec. II-B).
* ``merge``     -- Tikhonov normal equations (Eq. 2) with the Toeplitz form of
                   A*DA (Sec. II-C, the "type-1 with ones" kernel) and the direct
                   form, and a textbook conjugate gradient.
* ``mtip``      -- one slice -> match -> merge -> CG iteration on a sample.
* ``phasing``   -- error reduction, hybrid input-output and shrinkwrap on the
                   model's grid (Sec. II-D), with exact DFTs.

Parity status of each function is stated in its module header.
"""
