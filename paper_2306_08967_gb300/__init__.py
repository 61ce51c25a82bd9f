"""DAMF per-update hot path on one GB300 GPU (sm_103a): C ABI library + thin binding.

The compute runs in libdamf.so (hand-written CUDA, built in-tree by build.py); this
package only marshals arguments.  Importing it does not load the library; the first
DamfGraph does, and raises ImportError when the library has not been built.
"""

from .api import (DamfError, DamfFleet, DamfGraph, apply_edges_multi, batch_array, bytes_required,  # noqa: F401
                  core_svd, make_config, plan_slots, rsvd_width, step_multi)
