"""Condensed-space interior-point solver for box-constrained LQ-MPC on B300.

The compute path is liblqmpc.so (hand-written CUDA for sm_103a behind a C
ABI, declared in include/lqmpc.h); ``binding`` marshals arguments to it and
``inputs`` holds the seeded synthetic problem generators.  Importing this
package loads nothing; ``binding.load()`` opens the library.
"""

__all__ = ["binding", "inputs", "build"]
