"""GB300-native batched Flowtree (arXiv 1910.04126): C-ABI CUDA library + thin binding."""
