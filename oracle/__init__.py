"""FP64 CPU oracle of the D3Q19 BGK sparse-tile step (test infrastructure only)."""
