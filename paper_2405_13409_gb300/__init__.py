"""GB300-native specular-polynomial solver (CUDA library + thin binding)."""
