"""GB300-native triangular inversion by recursive triangular split (arXiv 2307.07611).

Importing the package loads nothing native; ``paper_2307_07611_gb300.lib`` loads the
CUDA library and fails loudly if it has not been built.
"""
