"""GB300 (sm_103a) FP64 hQR: recursive Householder QR of HODLR matrices
(Kressner & Susnjara, arXiv:1809.10585), behind the C ABI of include/hodlr_qr.h.

Every step of the factorization runs in the CUDA library; this package only builds it and
marshals arguments.  There is no CPU fallback: importing ``binding`` fails loudly when the
library is missing.
"""
__all__ = ["binding", "build"]
