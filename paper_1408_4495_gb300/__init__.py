"""GB300-native sparsifying-preconditioned Lippmann-Schwinger solver (arXiv:1408.4495).

The compute path is the C-ABI library ``libls`` (hand-written CUDA for sm_103a); this
package only marshals arguments to it (``paper_1408_4495_gb300.ls``) and provides seeded
synthetic workloads (``paper_1408_4495_gb300.workloads``).
"""

__all__ = ["ls", "workloads"]
