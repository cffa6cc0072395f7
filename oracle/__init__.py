"""FP64 CPU oracle for the pseudofermion HMC of the O(3) spin-fermion model
(Lunts, Albergo, Lindsey, arXiv:2204.14241).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the
CUDA library and imports nothing from it.

Everything here is plain numpy in float64 / complex128, written from the
paper's equations in the paper's index order and notation:

* fermion vectors have shape ``(2, 2, Nt, L, L)`` indexed ``[alpha, s, tau, x, y]``
  (band, spin, time slice, x, y), the order of Eq. (D_formula);
* the boson field ``phi`` has shape ``(3, Nt, L, L)`` indexed ``[a, tau, x, y]``
  (Section "Stochastic formulation of the determinant": phi as a 3 x Nt x L x L array);
* a set of ``k`` pseudofermion right-hand sides is a list of fermion vectors.

Modules
-------
``model``    parameters of the lattice model (Section "Sign-problem-free UV completion").
``fermion``  the fermion matrix D(phi) of Eq. (D_formula), dense and matrix-free, D^dagger, A = D D^dagger.
``boson``    the lattice boson action S_B and its gradient.
``solver``   CG and the twisted-Fourier preconditioned CG of Eqs. (Dsplit)-(precon).
``hmc``      pseudofermion heatbath, Fourier-diagonal metric, leapfrog, Metropolis, Eq. (covest).

Parity status: every function is pinned by a test under ``tests/`` against a closed
form, a symmetry the paper states, a library routine (dense solve) or finite differences.
Acceptance rates and physics observables are parity unpinned: the paper prints no
values for them.
"""

from . import model, fermion, boson, solver, hmc  # noqa: F401
