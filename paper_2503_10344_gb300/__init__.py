"""GB300 (sm_103a) PDLP: restarted, preconditioned PDHG for MIP LP relaxations.

The compute path is the CUDA library ``libpdlp.so`` (sources in ``csrc/``,
C ABI in ``include/pdlp.h``); :mod:`.binding` marshals arguments to it.
"""
from .binding import (FP_DUAL, FP_DUAL_FRAC, FP_FEASIBLE, FP_FRAC, FP_FRAC_DUAL, FP_FRAC_REDCOST,
                      FP_INFEASIBLE, FP_NODE_LIMIT, FP_NO_FINAL_LP, FP_REDCOST, FP_REDCOST_FRAC,
                      FP_STRATEGY, FP_TYPE, fp_run, fp_run_refs,
                      PDLP_FP32, PDLP_FP32_BF16A, PDLP_FP64, PDLP_ITER_LIMIT, PDLP_NUMERICAL,
                      PDLP_USED_BF16, PDLP_USED_PATTERN,
                      PDLP_OPTIMAL, PDLP_TIME_LIMIT, PDLP_PRIMAL_INFEASIBLE, PDLP_DUAL_INFEASIBLE,
                      DeviceLP, PdlpError, default_params, lib,
                      pdlp_polish_dual, pdlp_polish_primal, pdlp_solve, pdlp_solve_batch, pdlp_solve_batch_device, pdlp_solve_device,
                      pdlp_solve_device_noalloc,
                      time_kernels, time_kernels_batch,
                      workspace_size)
from .gnn import GnnGraph, GnnModel, pdlp_solve_warm, start_kkt

__all__ = ["FP_DUAL", "FP_DUAL_FRAC", "FP_FEASIBLE", "FP_FRAC", "FP_FRAC_DUAL", "FP_FRAC_REDCOST",
           "FP_INFEASIBLE", "FP_NODE_LIMIT", "FP_NO_FINAL_LP", "FP_REDCOST", "FP_REDCOST_FRAC",
           "FP_STRATEGY", "FP_TYPE", "PDLP_USED_BF16", "PDLP_USED_PATTERN", "fp_run", "fp_run_refs", "PDLP_FP32", "PDLP_FP32_BF16A", "PDLP_FP64", "PDLP_ITER_LIMIT", "PDLP_NUMERICAL",
           "PDLP_OPTIMAL", "PDLP_TIME_LIMIT", "PDLP_PRIMAL_INFEASIBLE", "PDLP_DUAL_INFEASIBLE",
           "DeviceLP", "PdlpError", "default_params", "lib",
           "pdlp_polish_dual", "pdlp_polish_primal", "pdlp_solve", "pdlp_solve_batch", "pdlp_solve_batch_device", "pdlp_solve_device",
           "pdlp_solve_device_noalloc", "time_kernels", "time_kernels_batch",
           "workspace_size", "GnnGraph", "GnnModel", "pdlp_solve_warm", "start_kkt"]
