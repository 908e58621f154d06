"""VB-QMC oracle: test infrastructure only (plain FP64 CPU restatement of arXiv:2207.14715, Sec. 2).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may import this.
"""
