"""FP64 CPU oracle for the RNN-wave-function VMC hot path (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code
with the CUDA path: it never imports ``paper_2507_18700_gb300`` and the CUDA
library never calls into it.

Every function is the plain definition the paper gives, written in numpy
float64, with loops over lattice sites and vectorisation over samples only:

* ``philox``      -- Philox4x32-10 counter-based generator (Salmon et al., SC'11)
* ``model``       -- 1D GRU (App. A), 2D GRU + GLU (App. A), softmax readout
                     (Eq. 3), autoregressive product (Eq. 1), sampling
* ``hamiltonian`` -- local energies of the TFIM (Eq. tfim) and of the
                     Marshall-rotated Heisenberg model (Eq. heisenberg) by full
                     re-evaluation of every connected configuration
* ``vmc``         -- energy statistics and the VMC gradient by an explicit
                     reverse sweep over the unrolled recurrence (Sec. III)
* ``growth``      -- the hidden-dimension embedding of Fig. 2(b)
* ``exact``       -- exact enumeration, exact diagonalisation and the
                     free-fermion ground energy used to pin the rest
"""
