"""B300-native limited first-order post-Newtonian N-body library.

The hot path -- the O(N^2) Newtonian + limited-1PN accelerations of one black
hole and N-1 stars (Tatekawa, arXiv:1801.07986, Section 2) inside a
kick-drift-kick leapfrog -- runs in hand-written CUDA kernels for sm_103a
behind the C ABI of ``include/pn.h`` (``libpn.so``).  :mod:`.pn` is a thin
ctypes binding with the same names; :mod:`.inputs` draws seeded synthetic
initial conditions.
"""
from .pn import (PN_FP64, PN_HERMITE, PN_KDK, PN_MIXED, PN_RK4, PN_PAIR_FUSED, PN_PAIR_TWO_PASS, PN_VHALF, PN_VPRED_END,  # noqa: F401
                 Context, PNError, pn_accel, pn_energy_noalloc, pn_init_batched,
                 pn_step_graph, pn_tune,
                 pn_accel_vjp, pn_destroy, pn_energy, pn_get_launch, pn_get_timing, pn_get_variant, pn_jerk,
                 pn_launch_count, pn_step_vjp, trajectory, pn_init, pn_last_error,
                 pn_set_params, pn_set_stream, pn_set_timing, pn_step, pn_step_host, pn_sync,
                 pn_version)
