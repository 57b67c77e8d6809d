"""FP64 CPU oracle for the MADmap PCG map-making solve (arXiv:0906.1775).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
float64 restatement of what the method computes, used to check the GPU
library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the library (``paper_0906_1775_gb300``) never
does, and this package imports nothing from the library.

Modules
-------
pointing   observed-pixel indexing and the sparse pointing matrix A, A^T
           (Section 3, Eqs. 1-4; Section 5.4)
noise      noise PSD, inverse-noise filter lags, banded block-Toeplitz N^-1
           (direct sum and circulant-embedded overlap-save FFT), FFT-length
           rule (Section 4, Eq. 13; Section 5.2, Eqs. 15-26; Appendix A)
solver     H = A^T N^-1 A, b = A^T N^-1 d, the block preconditioner, PCG with
           the lowest-residual output rule, and the dense Cholesky solve
           (Sections 3-5, Eqs. 8 and 10)
adjoint    gradient of a map loss through the solve by the implicit adjoint
multires   Q/U on a second pixelisation (Section 6, item 4)
gcp        pointing expanded from compressed boresight pointing (Section 5.3)
extended   extra columns [A B]: destriping offsets, binned templates and the
           half-wave-plate block (Section 6, items 1-3, Eqs. 39-43)

Every function carries "parity pinned by" notes naming the tests that tie it
to something other than itself.
"""

from . import pointing, noise, solver  # noqa: F401
