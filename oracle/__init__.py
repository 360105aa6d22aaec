"""Plain FP64 CPU oracle of the MLVS-DUGKS hot path.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library
under ``paper_2609_35258_b300/`` shares no code with it and never calls it.

Every function follows the paper step by step in numpy FP64 (summation over velocity in
ascending index order), citing the section / equation it restates:

* ``vspace``    -- Newton--Cotes velocity quadrature and the quadtree level spaces (Sec. 2.3, 3.1-3.2)
* ``kinetic``   -- reduced BGK/Shakhov model, moments, compatibility correction (Sec. 2.1, 3.3.1)
* ``dugks``     -- one DUGKS step on a structured Cartesian mesh (Sec. 2.2, Eqs. phi_update ... recover_phi)
* ``mapping``   -- hierarchical projection and moment-constrained mapping (Sec. 3.3.2)
* ``criterion`` -- contribution / transport criterion and hysteresis (Sec. 3.2)
* ``cluster``   -- mask decoding, graded distance, greedy clustering, enclosing masks (Sec. 3.2)
* ``curvi``     -- the DUGKS step on a structured curvilinear mesh (O-grid of the cylinder case, Sec. 4.4)
* ``mlvs``      -- multi-level step with cross-level faces (Sec. 3.4)
* ``mlvs_curvi`` -- the multi-level step on a structured curvilinear mesh (Sec. 3.4 on ``curvi``)
* ``unstructured`` -- the DUGKS step on polygonal cells (the two-cavity case of Sec. 4.5)
* ``mlvs_unstructured`` -- the multi-level step on polygonal cells (Sec. 3.4 on ``unstructured``)
* ``mlp``       -- FP64 reference MLP level selector (not in the paper; used to check gradients)

Functions without an independent pin say "parity unpinned" in their docstring.
"""
