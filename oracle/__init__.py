"""FP64 CPU oracle of the double-layer Jacobi method.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline and reference legs, never by the CUDA path.
"""
