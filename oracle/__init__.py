"""FP64 CPU oracle for time-step-targeting DMRG with Krylov time evolution.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` use it.  It shares no code with the CUDA path.

Alvarez, Dias da Silva, Ponce, Dagotto, "Time Evolution with the DMRG
Algorithm: A Generic Implementation for Strongly Correlated Electronic
Systems" (arXiv:1103.5391).

Modules
  ed            exact diagonalisation in the Fock basis (independent checker)
  blocks        exact block operators at a fixed left/right cut
  superblock    sector-pair H psi and excitation operators on the superblock
  krylov        Lanczos tridiagonalisation and the Krylov exponential (Sec. II.A, II.C)
  density       target weights and the weighted reduced density matrix (Sec. II.B, II.C)
  closed_forms  U=0 results of App. A and App. B, small-time expansion (Sec. III)
  models        exact chain and ladder problems at a fixed cut (blocks + superblock + ED labels)
  dmrg          textbook two-site DMRG (infinite + finite) of the Hubbard chain and two-leg ladder:
                truncated blocks, both wave-function transformations (Sec. I, Sec. II.B)
  tst           one finite sweep with time-step targeting (Sec. II.B-II.D, Eq. b)

Pins: tests/test_oracle_*.py; tests/test_oracle_mutations.py shows that planted mistakes in these
modules make the pins fail; tests/test_golden_fig2.py holds App. A's Fig. 2 curves against ED.

Every function is plain FP64 NumPy; a library primitive (matmul, eigh) may be
a step, but there is no blocking or fusion beyond the paper's definitions.
"""
