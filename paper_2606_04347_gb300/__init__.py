"""GB300 ETD step for the phase-field model of multicomponent membranes.

The compute path is the C-ABI library `libetd.so` (CUDA, sm_103a) built from `csrc/`;
this package only marshals arguments to it (see `abi`).  `workloads` builds seeded inputs.
"""
from .abi import Batch, EtdError, Plan, load_library, params_struct  # noqa: F401
