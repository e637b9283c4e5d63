"""GB300-native (sm_103a) Parareal/MGRIT shallow-water hot path (arXiv 2306.09497).

The compute path is the C-ABI library ``libswe_gb300.so`` built from
``csrc/``; :mod:`paper_2306_09497_gb300.swe` is the thin ctypes binding.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing (there is no CPU fallback).
"""
