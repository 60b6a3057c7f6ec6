"""GB300-native whole-body MPPI (arXiv 2409.10469): CUDA hot path behind a C ABI."""
