"""CPU oracle of the multi-level blended DG/FV scheme (Markert, Gassner & Walch,
"A Sub-Element Adaptive Shock Capturing Approach for Discontinuous Galerkin
Methods").

This package is TEST INFRASTRUCTURE. It is a plain, slow, FP64 numpy restatement
of the paper's method, written from its equations and algorithm sketches. Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import it. The product path (the CUDA library and its Python
binding) never imports, links or executes anything in here, and this package
shares no code with it.

Modules:
  ops          1D operators of one level (Sec. 2.1-2.5, eqs. fv-diff-matrix ...
               trafo-mv-nodal, the appendix on boundary evaluation operators)
  euler        Euler physics and the HLL flux with Einfeldt speeds (Sec. 3, 3.1)
  layout       element-major <-> global subcell grid layout conversion
  blended      the multi-level blended right-hand side (Sec. 2.5-2.7,
               appendix 3D extension and multi-level sketch)
  timestep     CFL time step (eq. cfl-condition) and SSP-RK3 stages
  plain_fv     independent first-order subcell FV scheme (pin for alpha = 0)
  plain_dgsem  independent nodal Gauss DGSEM (pin for alpha = 1 / forced levels)
  exact_riemann exact Riemann solver for the Euler equations (pin for Sod)

Pins (tests/test_oracle_*.py, run with -m "not gpu"): the operator identities of
Sec. 2.1-2.5, closed forms and tabulated Gauss rules, exactness on polynomials,
the surface-operator sparsity of the appendix, HLL consistency / wall / symmetry
properties, the exact Riemann star state against Toro's table, the alpha = 0 and
alpha = 1 limits against independent FV / DGSEM codes, forced intermediate levels
against sub-element DGSEM, free stream, conservation with random blending
factors, mirror / transpose / translation symmetry, the indicator on a ramp and
a step, design-order convergence and the Sod tube.

The blending factor inside the indicator's transition band is pinned by a
closed form: cubic profiles (along one axis, and the separable sum along both)
whose smoothness measures (total variations of the level polynomials) and
alpha = 0.5 are computed by hand from eqs. L1-norm-slope and calc-blending-factor.

The multi-D face blend of mixed-level elements (readings R1 / R2 in blended.py)
is pinned by a construction by hand: an element with two level-2 factors on its
two halves and data affine in rho (quadratic along x, linear along y), whose
inner-interface fluxes follow from the level polynomials' face values, the
weights (theta_L + theta_R) / 2 and numpy polynomial fits of the nodal fluxes.
"""
