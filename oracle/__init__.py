"""Plain FP64 CPU oracle of arXiv:1806.10247's cascaded LB step (test infrastructure only)."""
