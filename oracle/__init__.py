"""CPU FP64 oracle for junction-tree belief propagation.

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA path; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the C-ABI library and its Python binding) never imports, links or executes
anything here, and this package imports nothing from the product.

Contents:

* :mod:`oracle.hugin`   -- Hugin collect/distribute propagation (Eq. 1-3,
  Algorithms 2-4) in plain numpy FP64, plus the index mapping of Sec. 3.1.
* :mod:`oracle.brute`   -- enumeration of the joint distribution (the exact
  definition that propagation reaches), for tiny trees.
* :mod:`oracle.cpt`     -- clique tables from a Bayesian network's CPTs (the
  Initialization step of Algorithm 4).

Parity status of every function is stated in its module header: all are
pinned by ``tests/test_oracle_pins.py`` except where a header says
"parity unpinned".
"""
