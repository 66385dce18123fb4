"""GB300-native (sm_103a) hot path of the incompressible DUGKS with force term
(Wu, Shi, Chai and Wang, arXiv 1411.6121).

The compute path is the C-ABI library ``libdugks.so`` (hand-written CUDA kernels, see
``csrc/``); ``dugks`` is its thin Python binding. ``workloads`` holds the seeded
synthetic inputs. Importing the package does not load the library; ``dugks.load()`` does,
and fails loudly when the library has not been built.
"""
__all__ = ["dugks", "autograd", "workloads"]
