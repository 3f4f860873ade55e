"""FP64 CPU oracle for the sharing-ADMM hot path.

TEST INFRASTRUCTURE: imported only by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The CUDA library never imports, links or calls
anything here, and nothing here imports the library.
"""
from .sharing_admm import (Criterion, Eliminator, State, Result, RidgeSolver, sadmm, sadmm_primal_inverse, soft,
                           real_form, real_vec, forward, adjoint_re, objective, kkt, kkt_consensus, initial_state)
from .fista import fista, fista_consensus
from . import precision
from .signal_model import operator_from_delays, backprojection, db_image

__all__ = ["Criterion", "Eliminator", "State", "Result", "RidgeSolver", "sadmm", "sadmm_primal_inverse", "soft",
           "real_form",
           "real_vec", "forward", "adjoint_re", "objective", "kkt", "kkt_consensus", "initial_state", "fista", "fista_consensus",
           "operator_from_delays", "backprojection", "db_image", "precision"]
