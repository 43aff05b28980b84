"""Plain, slow CPU oracle for on-device network construction and spike delivery.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA path (``paper_2512_09502_gb300``), and the CUDA path
never imports it.

Every function follows one definition or method of the paper (arXiv 2512.09502) or of
a published method the paper relies on, cited in its docstring:

* ``philox``   -- Philox-4x32-10 (Salmon et al., SC'11), the counter-based generator
                  that replaces the paper's aligned RNG_{sigma,tau} streams.
* ``sampling`` -- integer-in-range, 24-bit uniform, Box-Muller normal, integer CDF
                  tables for quantised delays and Poisson counts.
* ``connect``  -- the connection rules (fixed in-degree, fixed total number,
                  pairwise Bernoulli) in generation order.
* ``layout``   -- per-rank source-sorted connection layout, image neurons and the
                  R/L/S/T/P (point-to-point) and H/I/G/Q (collective) maps.
* ``neuron``   -- iaf_psc_exp exact integration (Rotter & Diesmann 1999) and
                  ring-buffer spike delivery.

Floating point is fp64 throughout, except where a stored result is defined as fp32
(weights are rounded to fp32 once, as the paper stores them).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against values
the mathematics or a library routine fixes; see each module's header.  The network-
level spike trains are "parity unpinned": the dynamics are chaotic, so only their
statistics compare (as in the paper's own validation).
"""
from . import philox, sampling, connect, layout, neuron  # noqa: F401
