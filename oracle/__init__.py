"""Oracles for the Spectral Ewald Stokes library (TEST INFRASTRUCTURE ONLY).

* ``oracle.ewald``    -- the exact Ewald decomposition (C, FP64) that the method approximates.
* ``oracle.se_steps`` -- Algorithm 1 of the paper step by step in plain numpy (FP64).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may import
this package. The library under paper_2210_01255_gb300/ never imports it and shares no
code with it.
"""
