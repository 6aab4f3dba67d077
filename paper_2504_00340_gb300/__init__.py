"""GB300-native (sm_103a) depth-march solver for the linear-Boltzmann proton
pencil-beam model of arXiv 2504.00340.

The compute path is the CUDA library built from csrc/ (C ABI: include/pbs.h);
``binding`` marshals arguments to it, ``workloads`` makes seeded synthetic
inputs.  Importing this package loads neither torch nor the library.
"""

__all__ = ["binding", "build", "workloads"]
