"""Plain, slow FP64 CPU oracle for the SOAP density expansion of arXiv:2101.08814.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it. The product path (the CUDA library and its Python binding) never imports, calls or links anything
here, and this package imports nothing from the product path.

Each function writes out the plain definition from the paper, in FP64, with numpy:

  gto.py        GTO radial basis, its overlap matrix and the Löwdin S^-1/2 (Eq. GTO, Sec. 'GTO radial basis')
  hyp1f1.py     the restricted 1F1 function G(a,b,r) of Appendix A: series, asymptotic form, bisection switch,
                downward recurrences and dG/dr
  radial.py     the GTO radial integral (Eq. rad-int-gto-1), its derivative, the o-GTO transform, a direct
                quadrature of Eq. radial-integral-gaussian-density and the clamped cubic spline (Sec. 'Spline
                optimization')
  ylm.py        real spherical harmonics and their Cartesian gradients (Sec. 'Spherical Harmonics')
  neighbours.py brute-force periodic neighbour list (Appendix B's r_ji < r_cut over periodic images)
  soap.py       cutoff, density coefficients (Eq. spherical_expansion_coefficients_gaussians), power spectrum
                (Eq. nu2-basis-coupled), additive linear energy (Eq. additive-energy-model) and its gradients
                (Eqs. energy-derivative, energy-virial)
  mlp.py        a 1->H->H->F SiLU network with its backward pass and an Adam step, used to check the GPU
                training kernels of the learned radial surrogate

Every function is pinned by tests that do not reuse its own formula: quadrature, closed forms, special cases,
invariances, finite differences and library routines (scipy, mpmath) used only in tests.
"""
