"""Plain, slow FP64 CPU oracle of the MTF hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the ``libmtf`` C-ABI, its
CUDA kernels, the Python binding) may import, call or link this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path: the only common dependency is the input generator package
``mtf_inputs`` (meshes and plane waves, no method arithmetic).

Each function follows the paper (arXiv 2502.10907, "Local multiple traces
formulation for heterogeneous electromagnetic scattering"): section, equation
or algorithm numbers are cited in the docstrings.  Where the paper is silent
or inconsistent the reading taken is stated at the point of use.

Modules
-------
quadrature  Gauss-Legendre, symmetric 6-point triangle rule, Sauter-Schwab maps
skeleton    Algorithm 1 (subdomain spaces and normal swaps), RWG tables
operators   Galerkin EFIO/MFIO blocks, transmission Grams, incident data
mtf         MTF system of Problem 2, LU / GMRES solves, far field
mie         Mie series of a dielectric sphere (exact solution of Sec. 5.2)
brute       independent nested quadrature of singular pair integrals (pins)
osrc        block-OSRC preconditioner matrices (Sec. 4.4)
"""
