"""FP64 CPU oracle of the grand-potential phase-field lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow restatement of the
method of Verdier, Cartalade and Plapp (grand-potential phase field for a
two-phase ternary fluid with flow), written in float64 with plain PyTorch CPU
tensor operations and following the paper's equations in the paper's order.
Only the test suite, the package smoke check and the benchmark's CPU baseline
and reference arm may import it; the CUDA library never calls it and shares no
code with it.

Modules
  lattice  - D2Q5, D3Q7, D3Q19, D2Q9 velocity sets and weights (§3 tables, textbook sets)
  model    - thermodynamic closure, double well, interpolation, source (§2)
  lbm      - the coupled step with two-buffer pull streaming (§3; BGK, TRT or MRT flow)
  adjoint  - reverse-mode gradient of a final-field misfit (autograd through ``lbm``)
  analytic - closed forms used to pin the oracle (§2.4, §4.1, textbook decay laws)
  measure  - droplet count (union-find, Euler characteristic) and mean radius (§4.2.2)

Parity status: every function is pinned by a test in tests/test_oracle_*.py or
tests/test_workloads_and_measure.py except where its docstring says "parity
unpinned" (none does).
"""
