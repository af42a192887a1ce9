"""GB300-native digital backpropagation: single-step ESSFM and multi-step SSFM
(arXiv:1507.00921) as fused sm_103a CUDA kernels behind the C ABI in include/dbp.h."""
from .dbp import Batch, Plan, PlanInfo, describe  # noqa: F401
from ._lib import DBPError  # noqa: F401

__all__ = ["Batch", "Plan", "PlanInfo", "describe", "DBPError"]
