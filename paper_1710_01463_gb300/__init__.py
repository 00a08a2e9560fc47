"""GB300-native randomized truncated SVD (RSVD) for tensor-network bond compression.

Kohn et al., arXiv:1710.01463: Alg. RSVD (Sec. II.B) replacing full SVD + truncation
(Alg. TSVD, Sec. II.A) at every TEBD/DMRG-style bond update (Sec. III.A).

The compute path is librsvd.so (hand-written CUDA for sm_103a, C ABI in
include/rsvd.h); ``api`` and ``tebd`` marshal PyTorch CUDA tensors into it.
Importing this package does not load the library; the first call does, and
fails loudly if it was not built.
"""

__all__ = ["api", "tebd", "inputs", "build"]
