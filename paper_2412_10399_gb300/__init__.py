"""GB300-native compact-kernel MPM (CK-MPM) step: CUDA kernels behind a C ABI."""
