"""FP64 CPU oracle of the extended-matchgate probability path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline and reference legs, never by the library.
"""
from .extraferm_oracle import (  # noqa: F401
    CPHASE, GIVENS, PHASE, angle_layout, cphase_list, exact_amplitudes,
    estimate, exact_probabilities, expected_second_moment, extent, get_angles,
    prob_directional_derivative, prob_gradient, raw_estimate, sample_trajectories,
    sampling_probability, segments_and_layers, set_angles, splitmix64, trajectory_count_bound, trajectory_grid,
    wrap_angle,
)
from .philox import philox4x32_10, trajectory_uniforms  # noqa: F401
from .statevector import amplitudes as statevector_amplitudes, run_statevector  # noqa: F401
