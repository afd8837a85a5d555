"""GB300 runtime-adaptive equi-join (after "Eiger: An Efficient Library for
GPU-based Data Analytics").

The compute path is ``libeiger.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/eiger.h``); ``eiger`` is its Python binding and ``workloads``
draws seeded synthetic inputs.
"""

from . import eiger, workloads  # noqa: F401
from .eiger import (EigerError, Plan, Stats, join, join_into, join_sum, join_workspace,  # noqa: F401
                    load, plan, stats)
