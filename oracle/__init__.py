"""FP64 CPU oracle for the compressed FMM-FFT translation stage.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, NumPy implementation
of what the translation stage computes, written from the paper (Qian & Yucel,
"On the Compression of Translation Operator Tensors in FMM-FFT-Accelerated SIE
Simulators via Tensor Decompositions"), in float64 / complex128 throughout.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import it.  The product library never calls it, and it shares
no code with the CUDA path (the two meet only in ``seeded_inputs``, which holds
random-number generation and nothing of the method).

Modules
  directions  multipole count L, Gauss-Legendre x uniform direction grid (Sec. II.A)
  special     spherical Hankel h_l^(2) and Legendre P_l
  operator    translation operator (Eq. 7), near-field zeroing, circulant
              embedding, FFT'ed operator (Sec. II.A, Sec. II.B)
  fft         the oracle's own mixed-radix FFT
  translate   translation B = IFFT(T~ . FFT(A)) (Eq. 5) and its direct-sum twin
  decomp      Tucker-SVD (Alg. 1), H-Tucker-SVD (Alg. 2), TT-SVD (Alg. 3) and
              the per-direction restorations of Sec. II.C (Figs. 3, 4)
  pipeline    whole-stage drivers: operators for a plan, compression in the
              3D / 4D formats, compressed translation

Every function cites the passage of the paper it follows.  Parity status of
each function is recorded in its docstring; all are pinned by tests under
tests/ (no function here is "parity unpinned" except where stated).
"""
