"""CPU FP64 oracle for the ETD membrane step -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` may import or run anything in this package.  The CUDA product path never does,
and this package imports nothing from the product package; both sides take their inputs
from the seeded generators in `paper_2606_04347_gb300.workloads`, which hold none of the
method's arithmetic.

Contents (each module cites the passage it restates):
  fft        own mixed-radix FFT (forward unnormalised, inverse 1/N)
  spectral   folded wavenumbers, Laplacian symbol, l^phi, l^u, phi_0/1/2 (Sec. 2.2, 3.2)
  fd         D+-, Delta_{S,h}, Delta_h, central differences, <.,.>_h (Sec. 2.1)
  band       narrow band, components, band-restricted (-Delta_{S,h})^{-1} by CG (Sec. 3.2)
  model      W, g, f, R1, R2 (coupled and fixed), recovery, energy (Sec. 1, 3.1, Eq. (2.16))
  etd        ETD1/ETDRK2 spectral drivers, Algorithm 1 (Sec. 3.3)
  section2   dense variable-coefficient ETD of Sec. 2.2 (theorem checks, grids <= 32^2)

Pins (tests marked `not gpu`): brute-force DFT and numpy.fft for the FFT; series/quadrature/
multiprecision for phi_j; single Fourier modes (exact exponential); dense 8^2 matrix
exponentials by scipy.linalg.expm of augmented matrices (fixed step) and dense 8^3 ones for
one coupled ETD1/ETDRK2 step; the expansion identity R1 - L_phi phi = Eq. (1.1)/mu; the
line-tension, area and alpha terms of R1 on single-mode membranes in closed form; R2 (fixed,
and coupled without motion) as the negative L2 gradient of the discrete energy built from the
dense Sec. 2 matrices; model.energy against the dense Sec. 2 energy; the advection term on a
translated profile in closed form; FD identities (symmetry, summation by parts, discrete
eigenvalues); sparse direct solves for the band inverse; the maximum-bound and energy
theorems of Sec. 2.2 on dense grids; temporal orders of ETD1/ETDRK2.

Parity unpinned: the fully assembled coupled step over many steps (Algorithm 1 with R1, R2,
the advection and the band solve interacting) has no closed form or printed value; each of
its terms and one step of its driver are pinned as listed above.
"""
