"""Exact solutions the paper's test problems are compared against (Sect. "Sod
test", "Noh test", "Sedov test"): the Riemann problem of an ideal gas
(textbook iteration on the star pressure), the Noh implosion (closed form) and
the Sedov-Taylor blast (self-similar Euler equations).  These are references
for the physics of whole runs, not for the method's arithmetic: the tests pin
each against jump conditions and integrals, and use them to judge the
oracle's and the device's profiles; the benchmark uses the Riemann solution
for the L1 error of the batched ensemble.  Nothing here is called by the
library.
"""
