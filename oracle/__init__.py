"""Plain, slow FP64 CPU oracle for split-CTMRG of the triple-layer PEPS-PEPO-PEPS network.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link or execute
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code, headers, tables or
constants with the CUDA path; both sides only share the seeded input draw
(``paper_2506_19339_gb300/inputs.py``), which holds none of the method's arithmetic.

Modules (each function cites the passage of arXiv:2506.19339 it follows):

* ``ising``          -- Boltzmann weight W, sqrt(W), the Ising PEPO O (Sec. II, Sec. IV) and the
                        trivial identity PEPO used for the norm network <psi|psi>.
* ``bruteforce``     -- exact partition functions of tiny periodic lattices and exact
                        <psi|T|psi>, <psi|psi> on tiny tori (pins the network conventions).
* ``onsager``        -- Onsager's closed form for the 2D Ising free energy (a D=1 pin).
* ``split_ctmrg``    -- the split-CTMRG algorithm (Sec. III, Appendix) in the paper's order:
                        insertion/absorption, six projectors, renormalisation, convergence,
                        free energy (Eq. "free energy expression") and gradient (Eq. "gradient
                        expression").
* ``split_ctmrg_d2`` -- the D2-symmetric split-CTMRG (Sec. III.B, Eq. "Symmetry constraints"):
                        one projector set per iteration, corners absorbing a row and a column
                        at once, A and g projected onto the D4-invariant tensors.
* ``reduced_ctmrg``  -- the traditional reduced method (Sec. II, Fig. 3): an independent
                        reference algorithm for the same f and g.

Parity status: every function here is pinned by a ``-m "not gpu"`` test, except the
variational bound f(A) >= f_exact, which is "parity unpinned" (the paper prints no exact 3D
value to compare against).
"""
