"""GB300 (sm_103a) pseudo-potential D2Q9 lattice Boltzmann solver with the
geometric contact-angle wall rule (Hu, Li & Uddin, arXiv:1501.05430).

The solver is the C-ABI library liblbm.so (include/lbm.h) built from csrc/;
``paper_1501_05430_gb300.lbm`` binds it with the same names, and
``paper_1501_05430_gb300.inputs`` holds the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
from . import lbm  # noqa: F401

__all__ = ["lbm", "inputs"]
