"""FP64 CPU oracle for NFFT-accelerated Sinkhorn (Lakshmanan, Pichler, Potts,
"Nonequispaced Fast Fourier Transform Boost for the Sinkhorn Algorithm").

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the CUDA library and its Python binding) never imports,
calls or links anything here, and this package imports nothing from the
product: the two share no code.

Everything is plain numpy in float64, written to be checked against the paper
by eye:

* ``oracle.sinkhorn`` -- the Gibbs kernel, the exact kernel-vector products
  (Eqs. (matexp), (matexpt)), dense Sinkhorn (Alg. 1), the dual objective
  (Eqs. (14), (27)), the stopping residual (Eq. (Error)), the transport plan
  (Eq. (pi*)) and entropies (Eq. (negentropy), Lemma "Quality of the Sinkhorn
  approximation").
* ``oracle.fastsum`` -- the regularized periodic kernel (Sec. 4.1, "Regularization
  of K"), its Fourier coefficients b_k (Eq. (ansatz_NFFT)), the nonequispaced
  discrete Fourier sums and the fast-summation formula Eq. (fastsum) evaluated
  with exact trigonometric sums (no window, no FFT), plus the near-field
  correction for r = 1 (Remark "Arithmetic complexity").
* ``oracle.lp`` -- the Kantorovich linear program (Def. "Wasserstein distance",
  Eqs. (Da)-(Dd)) by brute force over permutations, for tiny inputs only.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and brute force; none is "parity unpinned".
"""
