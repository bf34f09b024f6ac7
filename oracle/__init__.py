"""FP64 CPU oracle of the TV-deblurring PCG path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this package. The CUDA library never does.
"""
from .tvd_oracle import *  # noqa: F401,F403
from .tvd_oracle import AR, R, PC_NONE, PC_DIAG, PC_FAST, PC_DFAST, PC_FASTD  # noqa: F401
from .tvd_oracle import METHOD_FP, METHOD_REBLUR, METHOD_REBLUR_ARL, REBLUR_METHODS  # noqa: F401
