"""FP64 CPU oracle of the discrete FIO (test infrastructure; see oracle.py)."""
