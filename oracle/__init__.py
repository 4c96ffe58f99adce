"""Plain, slow FP64 CPU oracle for the 3DPIFCM hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (``paper_2002_01981_gb300/csrc``); the
two meet only in the seeded input generator, which holds none of the
method's arithmetic.

Modules
-------
``oracle.ifcm``    Eqs 1-10 (objective, membership, centres, modified
                   distance, neighbourhood terms H and F, shell weights),
                   the FCM initialisation and the IFCM iteration loop.
``oracle.philox``  Philox4x32-10 counter-based generator (Salmon et al.,
                   SC'11) and the 53-bit uniform double built from it.
``oracle.pso``     Algorithm 1 steps 3-9 (particle swarm over (lambda, xi))
                   and the whole Algorithm 1 driver.
``oracle.precision``  bfloat16 rounding (nearest, ties to even) from the
                   format's definition, to model membership storage.
``oracle.adjoint`` reverse-mode dJ/d(lambda, xi) through K unrolled IFCM
                   iterations (Eqs 1-8 differentiated by the chain rule).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, hand-worked fixtures under
``tests/golden/``, brute force on tiny inputs, or published known-answer
vectors.  The absolute J and best (lambda, xi) on the synthetic phantoms are
"parity unpinned": the paper prints no worked example for them.
"""
