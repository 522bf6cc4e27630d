"""FP64 CPU oracle for the MLGMRES hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2103_10975_gb300``) never imports it and shares no code
with it; the only inputs both sides use come from the separate ``synthetic``
package, which holds none of the method's arithmetic.

Modules:
* ``native``  - plain-C restarted GMRES(m) with MGS and Givens rotations, the
                2D 5-point and 3D variable-coefficient 7-point operators.
* ``direct``  - dense assembly, DST-I fast Poisson solves, closed-form
                eigenpairs, brute-force Krylov least squares (the pins).
* ``nn``      - FP64 forward / backward / Adam of the initial-guess network.
* ``gate``    - Algorithm 1's moving-average gate, spread check and
                retraining counter.
* ``guess``   - the learned guess as a whole: c s N(b/s), then damped-Jacobi
                sweeps.

Parity status: the GMRES oracle, operators, network, guess and gate are each pinned
by tests under ``tests/`` against closed forms, dense LU, finite differences
or hand-worked sequences.  The online training trajectory as a whole is
parity unpinned (it depends on stochastic minibatch sampling); only its
per-step gradients and updates are pinned.
"""
