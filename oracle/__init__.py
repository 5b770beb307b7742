"""Plain FP64 CPU oracle of the patch-based AMR Euler solver (test infrastructure).

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. It shares no code with the CUDA library in ``paper_2508_05020_gb300``; the
two only read the same workload tables from ``synth``.

Modules
-------
euler     Euler equations, calorically perfect gas, characteristic projection,
          WENO5-JS nodal mid-point interpolation, Rusanov flux (Sec. 3, Eqs. 1-12),
          the HLLC flux option, the central schemes of Eqs. 8-9
mesh      patch hierarchy, R1/R2 rules, Algorithm 1 refinement closure and the
          Sec. 4.3 coarsening rule
amr       the solver around them: ghost fill, prolongation, boundaries, SSP-RK3
          stages, reflux, restriction, CFL step, refinement sensor, regrid
riemann   exact Riemann solver for shock-tube pins
mlp       FP64 refinement-indicator network (forward, backward, BCE, Adam)
flopcount instrumented FLOP count of the face flux and the cell update

Every floating-point expression is written in the evaluation order that the
FP64 GPU path uses (numpy evaluates each operator with IEEE rounding and never
fuses a multiply and an add), so the two can be compared bit for bit.

Parity status: every function is pinned by tests under ``tests/``, the
initial conditions included (shock relations, the printed implosion setup,
the double-Mach geometry, SplitMix64 reference outputs). The long-time
solutions of the Shu-Osher, four-quadrant, double-Mach and blast problems
have no closed form: there the pins are conservation, symmetry, uniform-fine
equivalence and the step-level pins (parity unpinned beyond those).
"""
