"""CPU FP64 oracle for the commutator-free exponential time-propagator (CFET).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of Alvermann & Fehske, "High-order commutator-free exponential
time-propagation of driven quantum systems" (arXiv:1102.5071), written in
numpy float64 / complex128.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it.  The CUDA product path never
imports, links or calls anything in here, and nothing in here calls the CUDA
path: the two share no code.

Modules
-------
schemes    coefficient tables f_{i,n} (Tables 1-5), the symmetric expansion
           rule R1 (Eq. FSymm), shifted Legendre polynomials (Sec. 3.1),
           Gauss-Legendre points/weights (Table 6) and g_{i,m} (Eq. OmGLeg).
operators  H v for the driven XXZ chain (Pauli-string definitions, Eq. 53-54
           style spin operators), the transverse field, general real sums of
           Pauli strings applied site by site, banded (DIA), compressed
           sparse row (CSR) and dense operators.
krylov     Lanczos / Krylov evaluation of exp(-i tau H) psi (Sec. 7.1) with
           the a-posteriori error estimate and time substepping.
cfet       the CFET time step (Eq. Ucf with Eq. OmGLeg) and time stepping
           (Sec. 6.1).
chebyshev  Chebyshev evaluation of exp(-i tau H) psi (the alternative technique
           of Sec. 8.1/8.2): Gershgorin intervals combined by Weyl's
           inequality, Jacobi-Anger coefficients, truncation by the Bessel
           tail bound, three-term recurrence; CFET stepping with it.
timestep   time-step selection (Sec. 6.6): error constant from two step
           sizes, the step for an accuracy goal, adaptive stepping by the
           per-step estimate.
interaction  CFET stepping in the interaction picture of the constant diagonal
           of H0 (Secs. 9.3, 9.4): stage operators sum_m g_{j,m} e^{i H_d t_m}
           H_b(t_m) e^{-i H_d t_m} applied by that definition.
adjoint    fidelity loss 1 - |<phi|psi(T)>|^2 of a CFET propagation with a
           piecewise-constant drive amplitude and its exact gradient (dense
           stage exponentials and Frechet derivatives; small systems).  The
           paper has no gradients: this is the plain definition.

Parity status: every function listed above is pinned by ``tests/test_oracle_*``
against closed forms or library routines, except the whole-pipeline result at
the driven-chain and grid-atom workloads, which no closed form covers; those
are pinned only through properties (factorisation at J=0, time-independent
exactness, order slopes, unitarity).  The gradient of ``adjoint`` is pinned by
central finite differences of its loss and by its vanishing at an optimum.
``operators.PauliSum`` is pinned by Kronecker products of the 2x2 Pauli
matrices, the XXZ chain written as strings, and the closed forms of
exp(-i t b Y) and exp(-i t J Y Y).  ``chebyshev`` is pinned by dense expm, the closed forms of the Sec. 8.2
harmonic-oscillator example and of the Jacobi-Anger series, and dense
Gershgorin intervals.  ``timestep`` is pinned by the driven two-level system's
exact propagator (predicted against true errors, goals met) and by the
time invariance of its local constant.  ``interaction`` is pinned by exactness
without off-diagonal terms, the resonant two-level system (constant
interaction-picture Hamiltonian, Eq. (TwoLevelU)), the order slope against
the Schroedinger picture and the dense stage operator.
"""

__all__ = ["schemes", "operators", "krylov", "cfet", "chebyshev", "timestep", "interaction", "adjoint"]
