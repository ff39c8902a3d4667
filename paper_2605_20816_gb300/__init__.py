"""GB300-native polynomial-diagram fitting (hand-written sm_103a CUDA behind a C ABI)."""
