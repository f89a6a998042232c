"""FP64 CPU oracle for the DD NM-ROM with hyper-reduction (arXiv 2305.15163).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA path: the library computes its own DD setup,
residuals, decoders and KKT solves; the two meet only at the seeded inputs from
``inputs/``.

Plain, slow and meant to be checked against the paper by eye: numpy / scipy in
float64, the formulas written in the paper's matrix notation.

* ``burgers``  -- Sec. 7.1: exact solution, centred-FD residual and Jacobian in the
  Kronecker form of Eq. (burgers_discretized), monolithic Newton (the FOM).
* ``dd``       -- Sec. 2: residual/interior/interface sampling, ports, compatibility
  matrices A_i (Eq. compatibility_conditions_mat).
* ``decoders`` -- Sec. 5.1/5.4: masked shallow decoder, its Jacobian, the HR subnet;
  Sec. 3.3: linear (LS-ROM) decoder and POD with the energy criterion.
* ``hr``       -- Sec. 3.1/5.3: gappy-POD hyper-reduction: residual snapshots from Newton's history,
  the residual POD basis, greedy row sampling, the projector (Z_i Phi_i^r)^+.
* ``autoencoder`` -- Sec. 5.1, 7.2-7.3: masked shallow autoencoders trained by mini-batch Adam.
* ``rom``      -- Sec. 3.1/4.1: WFPC DD-LSPG-ROM with collocation or gappy-POD HR, Gauss-Newton
  blocks, the KKT system Eq. (sqp_system) solved densely, Armijo backtracking on the
  norm of the KKT right-hand side, least-squares multiplier start, Eq. (relative_error).

Readings of points the paper leaves open are stated where they are used.
"""
