"""Plain FP64 CPU oracle for the VOF droplet-evaporation time step.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The CUDA library never
calls it, and it never calls the CUDA library: the two share no code.

The oracle follows Saufi, Frassoldati, Faravelli & Cuoci, "DropletSMOKE++: a
comprehensive multiphase CFD framework for the evaporation of multidimensional
fuel droplets" (arXiv 2005.02867), Sections 2 and 3, with the discrete readings
listed in the repository's design notes.  Every linear system is solved with a
sparse direct factorisation (scipy), i.e. to the exact discrete solution up to
rounding, so the oracle carries no iteration-count or tolerance choice.

Modules
  thermo  -- Clausius-Clapeyron, Raoult, Peng-Robinson Z / fugacities (Sec. 2.5)
  grid    -- uniform axisymmetric r-z or 3D Cartesian finite-volume metric
  step    -- initial state, one segregated time step (Sec. 3.1), diagnostics
"""
