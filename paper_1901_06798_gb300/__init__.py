"""GB300-native shallow-water AMR wave-propagation library (C-ABI + CUDA).

Importing the package loads nothing native; ``paper_1901_06798_gb300.binding``
loads the CUDA library and fails loudly when it is missing.
"""
