"""FP64 CPU oracle for the unbinned negative-log-likelihood hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product (the CUDA library and its Python binding) never imports, links or
executes anything here, and this package imports nothing from the product.

The GooFit 2.0 paper prints no formulas: it describes PDFs composed from basic
shapes by sum and product combination PDFs and fitted to unbinned datasets
(Fig. 1; Sec. 1), three-body amplitude PDFs (Sec. 1, Sec. 5), the time-dependent
four-body amplitude analysis (Sec. 5) and toy MC for normalisation integrals (Sec. 5).  Each function here therefore states the
textbook definition it implements, written out plainly in float64 with no
blocking, fusion or reordering; gradients come from PyTorch autograd of these
definitions.

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: closed forms vs scipy quadrature, incomplete-gamma identities, grid
factorisation, finite differences, kinematic identities, published RNG
outputs (numpy's Philox), and recovery of generated parameters within their
errors on toy fits.
"""
from . import pdfs, model, dalitz, fit, td4, td3  # noqa: F401
