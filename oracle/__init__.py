"""CPU complex128 oracle for exact tensor-network contraction (TEST INFRASTRUCTURE).

Only tests/, the package smoke check and bench.py's CPU-baseline leg may import this.
It shares no code with the CUDA library; both read the seeded inputs of `tn_inputs`.
"""
from .core import (contract, contract_slices, contract_one, slice_assignment,
                       restrict_leaves, step_costs, path_costs, Neumaier)
from . import pins

__all__ = ["contract", "contract_slices", "contract_one", "slice_assignment", "restrict_leaves",
           "step_costs", "path_costs", "Neumaier", "pins"]
