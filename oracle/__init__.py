"""FP64 CPU oracle for single-step ESSFM / multi-step SSFM digital backpropagation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The CUDA
product path never calls it, and it shares no code with the CUDA path: it has its
own DFT, FFT, physical-constant conversions, step table, overlap rule, receiver
and coefficient fit, all written plainly in float64 numpy from the paper
(Secondini et al., "Coherent 100G Nonlinear Compensation with Single-Step Digital
Backpropagation", arXiv:1507.00921):

* ``dft``        naive DFT (definition) and an own radix-2 FFT (Section III footnote).
* ``fiber``      beta2 / alpha conversions, effective length (Section II, after Eq. 2),
                 channel memory M (Section III), step table, overlap rule.
* ``dbp``        linear sub-step (Eq. 1), SSFM nonlinear sub-step (Eq. 2), ESSFM
                 nonlinear sub-step (Eq. 3), step chaining (Section II) and
                 overlap-and-save (Section III).
* ``link``       forward Manakov split-step channel simulator with EDFAs and ASE
                 (test-vector generator).
* ``rx``         matched filter, symbol sampling, data-aided gain, decisions, Q.
* ``fit``        coefficient optimisation by MSE (Section IV).
* ``adjoint``    reverse-mode gradient of the DBP chain.

Every function states the passage it follows.  Pins live in ``tests/test_oracle_*``.
"""
