"""GB300-native batched HNSW search (Hierarchical NSW, arXiv:1603.09320).

Importing the package loads nothing native; ``paper_1603_09320_gb300.hnsw``
binds the C-ABI library and fails loudly when it is missing.
"""
