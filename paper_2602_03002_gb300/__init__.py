"""GB300-native multi-depth ray casting with a depth-sensor model (RPL, Sec. 3.2.2, Algorithm 1).

Submodules:
  rpl        ctypes binding of librpl.so (same names as include/rpl.h) plus Scene / View owners
  build      in-tree nvcc build of librpl.so for sm_103a
  workloads  seeded synthetic scenes, robots, cameras and poses
"""
__all__ = ["rpl", "build", "workloads"]
