"""GB300-native GP fitness evaluation and subtree crossover (Langdon &
Banzhaf 2019, GPquick with AVX and pthreads), behind a C-ABI library.

Importing the package loads nothing native; `paper_1902_09215_gb300.gp`
loads the CUDA library on first use and fails loudly if it is missing.
"""
__all__ = ["synth", "gp"]
