"""Plain FP64 CPU oracle for the emRKC monodomain time step.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it; both sides receive the same seeded inputs from the
separate ``workloads`` package.

Contents, each following the paper step by step in float64:
  fem      P1 stiffness and row-sum lumped mass (Sec. 2.1, Eq. sd_sys)
  ionic    Hodgkin-Huxley, ten Tusscher-Panfilov 2006 (epi), a linear
           passive test model, and "none" (Sec. 2, Eq. monodomain)
  rkc      get_stages / get_coeffs / RKC_Iteration (Algorithm 1)
  emrkc    f_F, f_S, f_E split (Eq. mono_in_FSE), Exponential_Euler,
           Averaged_Force and emRKC_Step (Algorithm 3), run driver
  power    nonlinear power iteration compute_rho (Algorithm 5)
  reference  classical RK4 on f_F + f_S + f_E, and EXEX-RL / IMEX-RL
           (Algorithm 4)

Parity status: the TTP06 ionic model is "parity unpinned" beyond its rest
state and published single-cell action-potential characteristics; every
other function is pinned by closed forms, invariants or brute force in
tests/test_oracle_*.py.
"""
