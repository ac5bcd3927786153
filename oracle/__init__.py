"""FP64 CPU oracle of the Horseshoe-probit Gibbs sweep.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the sampler of Terenin, Dong & Draper, "GPU-accelerated Gibbs
sampling: a case study of the Horseshoe Probit model" (Sect. 5, Eq. 12 and the
update schedule that follows it), written in float64 numpy/scipy.  It exists to
check the CUDA library.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never calls it and
shares no code with it.

Modules
  philox  Philox4x32-10 counter-based generator and the counter map.
  tn      Truncated-normal draw by inverse CDF (and the paper's two-arm
          rejection sampler as an alternative mode for distribution tests).
  gamma   Cheng (1977) algorithm GB, 32 proposals per round, first accepted.
  sweep   State, initial values and one Gibbs sweep.
  fmt     Decoding of the stored X formats (bf16, fp8 e4m3 + column scales).
"""
from . import philox, tn, gamma, sweep, fmt  # noqa: F401
from .sweep import State, init_state, gram, sweep_once, run  # noqa: F401
