"""FP64 CPU oracle for the shrinking-domain particle-mesh step (Llinares 2017).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (``paper_1709_04703_gb300``); both
receive the same seeded inputs from ``paper_1709_04703_gb300.ics``, which
holds none of the step's arithmetic.

Modules
-------
cosmology   conformal time, lightcone distance chi(a), step schedule, growth
pm          one PM step in the paper's order (Table 2): drift, CIC deposit,
            source, Poisson solve (exact discrete solution by FFT / DST-I),
            gradient + CIC gather, kick, drift, lightcone shrink
pk          power spectrum estimator with CIC window and shot-noise correction

Every function is plain numpy/scipy in float64 and cites the passage of the
paper it follows.  Where the paper is silent the reading taken is stated in
the function's docstring.
"""
