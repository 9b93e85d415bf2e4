"""FP64 CPU oracle for local real-space RPA screening (Vinson & Shirley,
"Fast, efficient, and accurate dielectric screening using a local, real-space
approach").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test-suite, the smoke check and the CPU
baseline leg of the benchmark use it.  It shares no code with the CUDA
library; both sides consume the same seeded input arrays.

Every function is a plain, slow, obviously correct restatement of the paper,
in float64/complex128 NumPy:

  projection.project_direct   Eq. (bloch), Sec. VI.B method 1 (direct Fourier sum)
  projection.project_fft_lagrange
                              Sec. VI.B method 2 (FFT to the cell grid, 3rd-degree
                              Lagrange interpolation, Bloch phase)
  quadrature.*                Eq. (chi1) with the single-grid map of App. D.1
                              ("Energy integration"); mu mid-gap, zeta rule
  chi0.chi0_pairs             sum over occupied/unoccupied pairs implied by
                              Eq. (eq-rpa), Eq. (eq-green) and Eq. (chi1)
  chi0.chi0_green             the paper's own route: per-frequency Green's
                              functions (Sec. VI.D) multiplied and summed
  coulomb.coulomb_multipole   multipole form of v, Sec. VI.E
  dyson.screened_interaction  W = v + v chi0 W, Eq. (eq-reducible), (eq-W)
  induced.induced_potential   core-hole response in the (r, l, m) basis, Sec. VI.E,
                              with the short-range v1 of Eq. (eq-partition)
  alda.*                      ALDA vertex, Eq. (chi-alda) and (kxc_alda); density and
                              the exchange-only kernel of the uniform gas
  augment.augment             all-electron augmentation, Eq. (eq-aug1), (eq-aug2)
  grad.*                      analytic gradients of a scalar loss of W in pair
                              form (the paper has no gradients)

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: closed forms, brute-force numerical integration of Eq. (chi1), an
FFT evaluation of Eq. (bloch), invariants of chi0 and W, Sherman-Morrison
reductions of the Dyson equation and finite differences of the loss.
"""
