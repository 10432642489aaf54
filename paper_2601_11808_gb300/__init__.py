"""GB300-native streaming IVF-Flat index with slab-chained inverted lists
(after arxiv 2601.11808).  The compute path is the CUDA library
``libsivf.so`` built from ``csrc/``; ``sivf`` is its thin ctypes binding."""
