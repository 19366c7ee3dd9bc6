"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds *inputs only*: the model specifications of the five workloads
(structure, parameter truth values, observable ranges, kinematic masses) and
numpy-PCG64 generators of event samples.  It contains none of the fitting
method's arithmetic -- no density evaluation, no normalisation, no likelihood.
Samples are drawn with numpy's own distribution samplers plus range rejection;
where a sampler needs a density for accept--reject (the Dalitz model), the
caller passes that density in as a function.
"""
from .specs import (c1_spec, c2_spec, c3_spec, c4_spec, td3_spec, dalitz_resonances, DALITZ_MASSES, TD4_MASSES,
                    TD3_MASSES, TD3_RESONANCES, TD3_TRUTH,
                    TD4_AMPS, TD4_RESONANCES, TD4_TIME, param_names, param_values, observable_names, to_polar)
from .gen import (gen_c1, gen_c2, dalitz_box, dalitz_candidates, accept_reject, round_to_f32,
                  toy_sizes, gen_c4_candidates, four_body_phase_space, smear_times)

__all__ = [
    "c1_spec", "c2_spec", "c3_spec", "c4_spec", "td3_spec", "TD3_MASSES", "TD3_RESONANCES", "TD3_TRUTH", "dalitz_resonances", "DALITZ_MASSES",
    "param_names", "param_values", "observable_names", "gen_c1", "gen_c2", "dalitz_box",
    "dalitz_candidates", "accept_reject", "round_to_f32", "toy_sizes", "gen_c4_candidates",
    "four_body_phase_space", "smear_times", "to_polar", "TD4_MASSES", "TD4_AMPS", "TD4_RESONANCES", "TD4_TIME",
]
