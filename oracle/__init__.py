"""Plain CPU FP64 oracle of the method of Gatto & Hesthaven, "A Preconditioner
Based on Low-Rank Approximation of Schur Complements" (arXiv 1508.07798).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path (the
CUDA C-ABI library and its Python binding) never imports, calls or links it,
and it imports nothing from the product.

Every function follows the paper's definitions step by step in NumPy/SciPy
FP64, with no blocking, fusion or reordering beyond what the paper states:

  nd.py        Sec. 4.0 box tree and interior/boundary sets, eq. (30)/(31) order
  rademacher.py  counter-based +-1 test matrices (SplitMix64, published form)
  idecomp.py   interpolative decomposition, Sec. 2 (eq. 43 and its footnote)
  hss.py       randomized HSS construction, Theorem 1 (Martinsson 2011 scheme)
  factor.py    Algorithm 2 (leaf elimination, eq. (32) merge, eq. (36) top block)
  apply.py     the inverse factorization M^-t D^-1 L^-1 (end of Sec. 4.2)
  fgmres.py    restarted flexible GMRES with right preconditioning
  mlp.py       rank-prediction MLP of the learned-rank form (not in the paper):
               forward, loss gradient, Adam, standardisation
  ilu.py       block ILU(0), the comparison preconditioner of Sec. 5
  merge.py     structured merge (reading R2): eq. (37) block solve with the
               second Schur complement compressed (Algorithms 1 and 3)

Pins (tests/test_oracle_*.py): exact LDM^t with compression off equals a dense
LU solve; GMRES converges in one iteration then; ID error within the strong
rank-revealing bound of the SVD and |P| <= 2; HSS recovery of matrices that are
HSS by construction; Schur complement equals the inverse of the trailing block
of the front inverse; brute-force interior/boundary sets on tiny meshes;
unpreconditioned GMRES history equals SciPy's; ILU(0)'s product equals A on
A's pattern, is exact on a block-tridiagonal chain and equals scalar ILU(0);
the structured merge's block solve is the exact inverse of the interior block
perturbed by H~ - S~ (every parent and the top block).
"""
from .nd import nd_order                      # noqa: F401
from .idecomp import interp_decomp            # noqa: F401
from .hss import hss_tree_for_front, hss_compress, probe_residual, probe_threshold   # noqa: F401
from .factor import factor, box_schur, eliminate_front   # noqa: F401
from .apply import apply                      # noqa: F401
from .fgmres import fgmres                    # noqa: F401
from .rademacher import rademacher            # noqa: F401
from . import mlp                             # noqa: F401
from .ilu import ilu0, ilu0_apply             # noqa: F401
