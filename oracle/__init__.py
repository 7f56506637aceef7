"""Plain FP64 CPU oracle of the micromagnetic field/torque/DP45 path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or executes anything under `oracle/`; only
the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
use it.  It shares no code with the CUDA path: its own demag tensor, its own
stencils, its own Runge-Kutta stepper.  numpy's FFT is the one library
primitive it uses (for the zero-padded convolution).

Every function follows a passage of the paper (arXiv 2411.18194, "Methods"):
    demag.py    Magnetostatic field: Newell tensor below a cutoff, asymptotic
                expansion above it; B = -mu0 N * M with M summed over
                sublattices.
    fields.py   Exchange (Eq. AFM_exchange_field), interfacial DMI (Eq. dmi)
                with its Neumann boundary condition (Eq. AFM_Neumann_BC),
                uniaxial anisotropy, Zeeman, magnetoelastic field
                (Eq. magnetoelastic-field), LLG torque (Eq. LLG_torque).
    elastic.py  Elastodynamics (Eq. elasticity) with 4th-order central
                differences in the bulk, traction-free boundaries, and the
                magnetoelastic force (Eq. magnetoelastic-force).
    dp45.py     Dormand-Prince RK45 (Table of solvers) with FSAL and an
                adaptive step-size controller.

Parity pinned or unpinned: see the pins in tests/test_oracle_*.py.  The
adaptive-controller constants are a reading of a passage the paper leaves
open; they are agreed between the oracle and the CUDA path by construction
only ("parity unpinned").  The elastic edge stencils, also a reading, are
pinned by the exactness every row must have (linear and quadratic fields,
quartics in the bulk), the adjointness of the divergence, the absence of
growing modes and energy conservation.
"""
