"""GB300-native even-odd Wilson-clover Dirac operator and Krylov solvers.

The compute path is liblqcd.so (hand-written CUDA for sm_103a) behind the C
ABI of include/lqcd.h; ``lqcd`` is its thin ctypes binding.  Import
``paper_1103_1363_gb300.lqcd`` to use it (it raises if the library has not
been built with ``__graft_entry__.build()``).
"""
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblqcd.so")
INCLUDE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
