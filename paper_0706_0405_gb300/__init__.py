"""GB300-native (sm_103a) KT D2V9 finite-difference lattice Boltzmann step with
the added dissipation term of Pan, Xu, Zhang & Jiang (IJMPC 2007).

The compute path is the CUDA library ``liblbm.so`` (sources in ``csrc/``,
C-ABI in ``include/lbm.h``); ``lbm`` is its ctypes binding and ``workloads``
states the synthetic problems.  Importing this package loads nothing; the
library is opened on first use of ``lbm``.
"""
