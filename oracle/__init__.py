"""Plain FP64 CPU oracle for the entropy-stable van der Waals moving-mesh scheme.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no common kernels, headers, helpers or constant
generators) and imports nothing from the ``paper_2407_05568_gb300`` package.

It is written for a reader who checks it against the paper by eye: numpy
arrays in float64, whole-array operations that follow the formulas in the
paper's order and notation, no blocking, fusion or reordering beyond what the
formulas state.  Every function cites the section / equation it follows.

Modules
  thermo   -- van der Waals EOS, sound speed, fundamental derivative, entropy
              variables and potentials (Sec. 1, Sec. 2, Def. 2.1)
  ecflux   -- logarithmic mean and the two-point EC flux (Sec. 3.1,
              eq. (ECCondition_comp), Theorem 3.1 and the explicit solution)
  weno     -- fifth-order multi-resolution WENO reconstruction (Sec. 3.3)
  operator -- metrics (eq. SCLCoeff, VCLCoeff), high-order EC flux
              (eq. ECFlux_curv_2p, GCL_flux), ES dissipation (eq. HOstable),
              the semi-discrete right-hand sides (eq. semi_U, semi_J)
  mesh     -- monitor, low-pass filter, Jacobi sweeps, limiter (Sec. 4)
  stepper  -- CFL time step (eq. cfl) and SSP-RK3, one full time step

Parity status of each part is listed in ``PINS`` below; "unpinned" parts are
those where the paper gives no value or closed form to check against.
"""

PINS = {
    "thermo": "pinned: Table 5.1 G values, critical point, ideal-gas limit",
    "ecflux": "pinned: consistency, symmetry, Tadmor condition, paper's units-B formula",
    "weno": "pinned: linear-weight limit equals the 5-point value, constants, design order; "
            "parity unpinned for the nonlinear weights (cited MR-WENO reference not in the paper)",
    "operator": "pinned: discrete SCL, free stream, entropy conservation of the EC scheme, "
                "entropy production sign of the ES scheme, eigen-system identities",
    "mesh": "pinned: filter preserves constants and sums, uniform monitor fixed point, "
            "1D equidistribution; parity unpinned for boundary handling (paper silent)",
    "stepper": "pinned: SSP-RK3 order on an ODE, design order on smooth advection, "
               "free stream on a moving mesh",
}
