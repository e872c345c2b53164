"""NFFT-accelerated Sinkhorn on GB300 (sm_103a CUDA behind a C ABI)."""
