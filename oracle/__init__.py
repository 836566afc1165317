"""FP64 CPU oracle of the deflated restarted Lanczos methods (test infrastructure).

This package is the plain, slow, obviously correct reference that the CUDA
path is checked against.  It is test infrastructure: only the tests, the
package smoke check and the benchmark's CPU-baseline leg may import it.  It
shares no code with the CUDA library and never imports it.

Contents, each following the paper (arXiv:0901.3163, Abdel-Rehim, Morgan,
Nicely, Wilcox) where the paper fixes the method:
  wilson  -- the Wilson matrix M, M^dagger M and gamma5 M (Sec. 2), NumPy;
  cwilson -- the same Wilson matrix as plain C loops (speed for big lattices);
  krylov  -- CG and MinRes (Sec. 1), the Lanczos recurrence, Lan-DR(m,k) and
             MinRes-DR(m,k) (Sec. 1, Sec. 2), D-CG and D-MinRes (Sec. 2);
  kappa   -- the kappa rule of the synthetic workloads (min|eig(gamma5 M)|);
  evenodd -- the even-odd (Schur complement) form of M on the even sites (not
             in the paper; the standard reduction the deflated methods apply to).

The paper defers the definition of the four deflated algorithms to its
ref. [3]; what is written here is the standard thick-restart reading
(regular Ritz vectors + Galerkin solve for Lan-DR, harmonic Ritz vectors +
minimum-residual solve for MinRes-DR), stated step by step in each docstring.
"""
