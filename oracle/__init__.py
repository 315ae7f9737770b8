"""FP64 CPU oracle of the DEM timestep (test infrastructure only)."""
