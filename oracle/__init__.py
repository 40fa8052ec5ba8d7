"""Plain FP64 CPU oracle of the ADER-DG Navier-Stokes scheme (Krenz, Rannabauer,
Bader, arXiv 1905.05524, Sections 2 and 3).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` (as the checker) and
by ``bench.py``'s CPU baseline leg.  It shares no code with the CUDA library
(its own basis construction, physics, predictor, corrector, indicator and
adjoint), and it never reads a value produced by the CUDA path.

Everything is written for readability, not speed: plain PyTorch CPU tensor
operations in float64, vectorised over cells only, with ``torch.einsum`` as
the single library primitive for the small tensor-product contractions.

Parity status per function (which test pins it) is listed in the module
headers.  Functions whose constants the paper does not fix are marked
"parity unpinned" there.
"""
import torch

DTYPE = torch.float64
