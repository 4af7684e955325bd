"""GB300-native factor/solve of optimal-control KKT systems (Cyqlone-style segment
Riccati recursion + cyclic reduction), behind a small C-ABI CUDA library."""
