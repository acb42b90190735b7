"""GB300-native exact nearest-neighbour DTW retrieval cascade.

Implements the cascade of D. Lemire, "Faster Retrieval with a Two-Pass
Dynamic-Time-Warping Lower Bound" (arXiv:0811.3301): warping envelope,
LB_Keogh, LB_Improved and band-constrained DTW_p with early abandoning,
linked by best-so-far pruning, as hand-written CUDA kernels for sm_103a
behind the C ABI of include/dtwknn.h (libdtwknn.so).

`from paper_0811_3301_gb300 import api` loads the library and fails if it
is not built (`python -m paper_0811_3301_gb300.build`).
"""
