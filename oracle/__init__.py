"""CPU oracle of the 8x8 approximate-DCT block codec (arXiv 1808.02950).

TEST INFRASTRUCTURE.  This package is the plain, slow, independent reference
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the package
``paper_1808_02950_gb300`` and its CUDA library) never imports, links or
executes anything here, and this package never imports the product.

Modules
-------
matrices   -- exact DCT, T1/T2 and the literature matrices, factors of T1
measures   -- figures of merit of Tables 5 and 6
search     -- the greedy angle search of §3 (Eq. (6), Fig. 1)
codec      -- the blockwise codec of §6.1 (C, int64 / FP64) + Fraction brute force

Parity status: every function is pinned by a ``-m "not gpu"`` test against
values the paper prints or against closed forms / brute force; none is
"parity unpinned" except the image-level PSNR values themselves, which the
paper reports only for images that are not available here.
"""
