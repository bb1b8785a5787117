"""CPU ORACLE for fast polynomial evaluation -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU restatement of Algorithm A_p of
Anton, Mihalache and Vigneron, "Fast Evaluation of Real and Complex
Polynomials" (arXiv 2211.06320): exact scales and concave cover, the good
index set G_p, the per-point windows, and extended double-double Horner
sums.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import, call or link it.  It shares no code with the CUDA
path and never imports it.
"""
from .fpe_oracle import (NEG_INF, ExtValues, Preconditioned, concave_cover, cover_value, fpe_eval,
                         fpe_eval_fp64, good_mask, horner_ref, log2_abs, num_threads, offset_T, precondition,
                         scale, scale_of_int, set_threads, window_sum, window_sum_fp64, windows,
                         windows_bruteforce)

__all__ = ["NEG_INF", "ExtValues", "Preconditioned", "concave_cover", "cover_value", "fpe_eval", "fpe_eval_fp64",
           "good_mask", "horner_ref", "log2_abs", "num_threads", "offset_T", "precondition", "scale",
           "scale_of_int", "set_threads", "window_sum", "window_sum_fp64", "windows", "windows_bruteforce"]
