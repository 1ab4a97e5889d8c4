"""GB300-native spin-1/2 FTLM hot path: S^z-sector Heisenberg H.v gather, the Lanczos
recurrence around it and the FTLM trace estimator (arxiv 2605.26261).

The compute path is the CUDA library ``libftlm.so`` behind the C ABI declared in
``include/ftlm.h``; ``paper_2605_26261_gb300.ftlm`` is its thin Python binding.
``paper_2605_26261_gb300.inputs`` builds synthetic inputs (graphs, grids, vectors).
Importing the package does not load the CUDA library.
"""
