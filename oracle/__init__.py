"""CPU complex128 oracle for the Born-preconditioned Helmholtz hot path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library
(``paper_2603_18527_gb300``) never does, and it never imports the library.  It
shares no code with the CUDA path: only the seeded input recipes in ``synth/``
serve both.

Everything is float64 / complex128 on the CPU, written with plain PyTorch CPU
ops (``torch.fft`` as the FFT step, ``conv2d`` as the convolution step) so that
each function can be read against the paper's equations:

* ``helmholtz``: the Fourier pseudospectral discretisation (App. Fourier
  Pseudospectral Discretization), the split A = L_eta - V_eta (Eq. A_split),
  the Green operator G_eta by FFT, the CBS iteration (Eq. CBS), the NPBS
  iteration (Eq. npbs_integral) and its left-preconditioned form
  (Eq. npbs_iter), the stopping rule rTol (Sec. 5), and the adjoint operators.
* ``fgmres``: restarted flexible GMRES (the paper's FGMRES comparison, Sec. 5.1.3,
  after Saad 1993) on the Lippmann-Schwinger system (Eq. LS_discrete).
* ``unet``: the residual-to-correction U-Net (App. Experimental Setup, U-Net
  backbone) and the metric-matched unrolled loss (Eq. L_bs_Reta_integral).
* ``dense``: explicit dense matrices of the same operators for tiny grids,
  built from the DFT definition (no FFT), used only to pin the above.

Pins (``tests/test_oracle_pins.py``, ``tests/test_oracle_unet.py``) tie each
function to something other than itself: dense matrices from the DFT
definition, closed forms, algebraic identities, brute force and central finite
differences.  ``tests/oracle_mutation_check.py`` plants plausible mistakes in a
copy of this package one at a time and requires each to fail a pin.

Parity unpinned: nothing here depends on the paper's trained weights or on
OpenFWI; the trained network's iteration counts are reported, not pinned.
"""
