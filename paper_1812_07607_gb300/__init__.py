"""GB300-native exact epsilon-similarity join and top-k join over patch features.

The compute path lives in the C-ABI library built from `csrc/` (see
`include/dl.h`); `paper_1812_07607_gb300.dl` is the thin ctypes binding to it.
Importing this package does not load the library; `workloads` only draws inputs.
"""
