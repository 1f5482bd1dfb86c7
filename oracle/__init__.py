"""The oracle: test infrastructure only.

A plain, slow FP64 CPU CT-AUX walker (``ctaux_oracle.c``), an exact
diagonalisation of small Hubbard clusters (``ed.py``) and a builder for the
bare isolated-cluster propagator (``g0.py``).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import anything from this package; the GPU library
and its Python binding never do.
"""
