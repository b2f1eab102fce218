"""B300-native batched Paillier and private distributed ADMM (3P-ADMM-PC2).

The compute path is the C-ABI library ``libpc2.so`` (hand-written CUDA for
sm_103a); ``paper_2601_14980_b300.pc2`` is its thin ctypes binding.  Importing
the package itself loads nothing, so the seeded input generators in
``workloads`` stay usable on machines without a GPU.
"""
