"""B300-native BOLT oblivious map (Guo et al., CCS '25): CUDA kernels for
sm_103a behind a C ABI (include/bolt.h), with a thin ctypes binding."""
