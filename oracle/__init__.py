"""Plain FP64 CPU oracle for the QTT denoising-convolution path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path: it is written from the paper (arXiv 2301.13339, "Denoising
Convolution Algorithms and Applications to SAR Signal Processing") with numpy
and LAPACK (via numpy) as its only primitives, in float64 / complex128.

Modules
-------
``qtt``      -- QTT reshape (Sec. 4), TT-SVD (Alg. 1 + the max-rank
                modification of Sec. 5), Full (Alg. 3), TT-rounding,
                interleaved 2D bit order.
``conv``     -- the discrete linear convolution of Eq. (dconv) by direct
                sums and by zero-padded FFT (Sec. 2), the sinc imaging kernel
                of Eq. (GAF) / Eq. (sinc_kern1), the E_2 error (Eq. err_conv).
``toeplitz`` -- the QTT Toeplitz operator of the sinc kernel, operator x
                vector core contraction.
``pipeline`` -- decompose -> convolve in QTT -> round -> full (Alg. 2 with the
                Toeplitz convolution step), and the deconvolution loss, its
                dense adjoint and its core gradients.
``rsvd``     -- the range finder and randomized SVD (App. A, Algs. 4-5) and the
                max rank TT-RSVD (Sec. 5 modification (2)).
``qfft``     -- QTT-FFT / QTT-iFFT (Sec. 4, truncated as in Sec. 5), the
                Hadamard product and the QTT convolution of Alg. 2 Step 3.
"""
from . import qtt, conv, toeplitz, pipeline, rsvd, qfft  # noqa: F401
