"""GB300-native differentiable Projective Dynamics (DiffPD, arXiv 2101.05917).

The compute path lives in the native library libdiffpd.so (CUDA, sm_103a) behind
the C ABI of include/diffpd.h; this package only binds it (`_native`), gives it
a PyTorch front end (`api`, `autograd`) and builds it (`build`).
"""
from . import build  # noqa: F401
