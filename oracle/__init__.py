"""CPU oracle for the multiple-precision complex GEMM (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from here.
The product path (``paper_2307_06072_gb300``) never does: it fails loudly
when its CUDA library is missing instead of falling back to the CPU.

* ``exact``      O1 in Python: the exact triple loop (Eqs. 4m_way_base /
                 3m_way_base) and one round-to-nearest-even to p bits.
* ``c_oracle``   O1 in C (OpenMP), the same definition for large sizes.
* ``ozaki``      O2: the Ozaki split / slice products / exact accumulation of
                 Algorithm 2 in this library's integer reading, step by step,
                 used to check the CUDA path's integer stages bit for bit.
"""
