"""GB300-native lattice Boltzmann for moving rigid spheroids.

The method (D3Q19 lattice Boltzmann, link bounce-back on moving ellipsoids,
momentum exchange, implicit velocity and quaternion update) runs in
liblbsph.so, hand-written CUDA for sm_103a behind the C ABI of
include/lbsph.h.  This package is its build step and its Python binding.
"""
from .lbsph import (LB_BF16, LB_FIELD_DF, LB_FIELD_F, LB_FIELD_RHO, LB_FIELD_SOLID, LB_FIELD_U,  # noqa: F401
                    LB_FP16, LB_FP32, LBError, Simulation, lb_abi_version, lb_create, lb_destroy,
                    lb_get_drag, lb_get_fields, lb_get_force_torque, lb_get_force_torque_async, lb_get_links,
                    lb_last_error,
                    lb_lattice, lb_lattice_q, lb_profile_step, lb_set_external, lb_set_particles, lb_status_string, lb_step, lb_step_io,
                    lb_synchronize, library)
