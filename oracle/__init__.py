"""Plain FP64 CPU oracle for the multi-shifted BiCG RIXS path.

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct restatement
of what the method computes, written from the paper's equations.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import it;
the library and its Python binding never do, and they share no code with it.

Modules
-------
hubbard   occupation-number basis, fermionic operators with an explicit
          Jordan-Wigner sign, the Hubbard Hamiltonian H (Eq. 9) and the
          core-hole Hamiltonian H' (Eq. 10) as CSR matrices, and O1 / O2.
solvers   ground state by Lanczos, independent per-shift solves of Eq. (A1)
          (sparse LU and BiCGStab), the MSBiCG recurrences of App. C / Alg. 1
          in corrected form, and a full dual-space BiCG (App. A).
spectrum  the second step of Eq. (1): Lanczos continued fraction, direct
          solves at every loss energy, and the Lehmann (Kramers-Heisenberg)
          sum by full diagonalisation.
rixs      the whole map I(w_in, w) of Eqs. (1)-(2) assembled from the above.

Parity status of each function is stated in its module header; every function
listed there is pinned by a `-m "not gpu"` test against a closed form, an
invariant, full diagonalisation or a library routine.
"""
