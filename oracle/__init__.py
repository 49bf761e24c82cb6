"""Plain FP64 CPU oracle for randomized block matrix multiplication (Niu & Li).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

Each function cites the passage of the paper it follows.  Floating point is
FP64 throughout (numpy), integers that decide sampling are exact Python /
numpy unsigned integers.  Library primitives (matmul, sums, searchsorted)
serve as single steps; there is no blocking or fusion.

Modules
  stats      -- column/row norms, per-block statistics, exact ||M^k N_k||_F^2
  design     -- sampling probabilities (eq. 1.2, 1.4, 3.8, uniform) and
                block sizes (eq. 3.9, 4.2, 4.7, c/K) with integer apportionment
  sampler    -- Philox4x32-10 counter RNG and the fixed-point inverse CDF
  estimator  -- Alg. 1/2/3 estimators, block sampling, closed-form expected
                errors (Lemma 2.1, Remark 2.2, eq. 3.10), bounds (eq. 3.11,
                4.3) and the adjoint of the sampled product
  errors     -- error bars: per-entry variance (eq. 3.7, Thm 3.1), its
                one-sample estimate from the draws, and the whole-matrix
                report (Remark 2.2, eq. 3.10-3.12, 4.3-4.4, 4.8-4.9)

Pins (see tests/test_oracle_*.py): library norms and products, brute-force
enumeration of every sampling outcome on tiny inputs (exact expectation and
exact squared error), optimality of eq. 3.8/3.9 by perturbation, an
exact-rational highest-averages apportionment, an independent Philox
implementation, exact interval counts of the inverse CDF, Monte Carlo against
the closed form, finite differences for the adjoint.

Parity unpinned: the integer apportionment rule and the draw-to-counter
convention of the sampler are conventions of this implementation (the paper
states neither); they are pinned only through invariants and equivalences,
not against numbers printed in the paper (it prints none).
"""
from . import stats, design, sampler, estimator, errors  # noqa: F401
from .stats import *  # noqa: F401,F403
from .design import *  # noqa: F401,F403
from .sampler import *  # noqa: F401,F403
from .estimator import *  # noqa: F401,F403
from .errors import *  # noqa: F401,F403
