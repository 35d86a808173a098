"""FP64 CPU oracle for the AD-census matcher of arXiv 2203.02300 (Sect. 4).

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this package.  It shares no code with the CUDA
library in paper_2203_02300_gb300/ and neither imports the other.

Parity-pinning status of each function is listed in oracle/oracle.py's
docstring and in the test files that pin it.
"""
