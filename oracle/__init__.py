"""FP64 CPU oracle for the CK-MPM step: test infrastructure, never imported by the product path."""
