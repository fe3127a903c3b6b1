"""GB300-native brute-force dedispersion and single-pulse search.

The compute path lives in a C-ABI shared library (``libaa_gb300.so``, built
from ``csrc/`` for sm_103a); this package only binds it.
"""
