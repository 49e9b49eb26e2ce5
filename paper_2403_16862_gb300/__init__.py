"""GB300-native (sm_103a) hot path of INPC's implicit point cloud.

Stages (each a hand-written CUDA kernel behind the C ABI in include/inpc.h):
octree point sampling, multi-resolution hash-grid query and the
differentiable bilinear point rasterizer (forward and backward).
"""
