"""FP64 CPU oracle for the plane-wave Fock exchange operator (test infrastructure only)."""
