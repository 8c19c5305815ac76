"""FP64 CPU oracle of the fractional-step FV / immersed-boundary time step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA path (``paper_2505_23940_b300``) and never
imports it.

Everything is written with plain ``torch.float64`` CPU tensor ops, vectorised
over the grid but with no blocking, fusion or reordering beyond what the
paper's equations state.  Because it is plain tensor code, ``torch.autograd``
through ``step()`` gives the exact discrete adjoint of the oracle's own step;
that is the oracle of the hand-written adjoint (the paper differentiates its
solver the same way, by reverse-mode AD, §2.4.1).

Modules
  grid     staggered (MAC) finite-volume grid and metrics (§2.3.1)
  fluid    convection-diffusion operator, divergence, gradient, BCs (§2.3.1)
  poisson  exact solve of the discrete pressure Poisson equation (Eq. 9)
  ib       delta kernels, solid / IB classification, interpolation and force
           spreading (§2.3.3, Eqs. 18-23)
  body     rigid-body oscillator with RK4 (§2.3.2, Eq. 12)
  step     one fractional-step time step (Eqs. 4-10) with FSI coupling

Parity status per function is recorded in each module's header.  Functions
without an independent pin say "parity unpinned".
"""
from .grid import Grid, PERIODIC, NOSLIP, FREESLIP, INFLOW, OUTFLOW  # noqa: F401
from .step import State, step, kinetic_energy  # noqa: F401
