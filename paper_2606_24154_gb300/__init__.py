"""GB300-native neBEM hot path: closed-form influence of flat rectangular and
triangular boundary elements (with periodic images), influence-matrix fill, dense
LU solve, potential/field evaluation and space-charge direct sums, behind the
C-ABI library ``libnebem`` (see ``include/nebem.h``).

The binding is loaded lazily: ``from paper_2606_24154_gb300 import nebem``.
"""
__version__ = "0.1.0"
