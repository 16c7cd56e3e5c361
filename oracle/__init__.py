"""FP64 CPU oracle for SketchNE (test infrastructure only; see sketchne_oracle)."""
